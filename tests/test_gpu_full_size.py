"""GPU parity at the benchmark's full sizes, in the configurations the
benchmark times, on outputs that can be checked one by one: sampled rows of
X against the closed-form inverse each generator builds from its factors,
plus the Penrose / Drazin residuals computed on the device.  (The oracle's
iteration is not row-separable, so at these sizes the closed form is the
reference; the smaller parity tests compare with the oracle directly.)

Tolerances: 1e-9 relative for FP64-finished solves, 1e-4 for FP32-finished
ones (the bars the workloads are specified with)."""

import numpy as np
import pytest

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


def test_moore_penrose_4096x3072_as_benchmarked(handle):
    """Rank 2304, s log-spaced in [1e-4, 1]; FP64-class products, stabilised
    after a step below 0.5, order-18 stop at 1e-2, cleanup finish."""
    w = W.rectangular(4096, 3072, 2304, 1.0, 1e-4, seed=1)
    alpha = 2.0 / (w.s[0] ** 2 + w.s[-1] ** 2)
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp64_tc",
                           variant="stabilized", switch_tol=0.5, finish="clean", check=True)
    assert info["status"] == 0
    rows = np.random.default_rng(0).choice(3072, 32, replace=False)
    assert rel(X.cpu().numpy()[rows], (w.V[rows] / w.s) @ w.U.T) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_moore_penrose_4096x3072_mixed_schedule_as_benchmarked(handle):
    """The benchmark's loop-schedule arm: FP32-class loops while the iterate
    grows, then FP64-class loops (the last one stabilised), alpha = 1/s_1^2,
    order-18 stop, cleanup finish in FP64 class."""
    w = W.rectangular(4096, 3072, 2304, 1.0, 1e-4, seed=1)
    alpha = 1.0 / w.s[0] ** 2
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp32",
                           variant="stabilized", switch_tol=0.9, finish="clean", check=True)
    assert info["status"] == 0
    assert 3 in info["precision"] and info["precision"][-1] == 4
    rows = np.random.default_rng(0).choice(3072, 32, replace=False)
    assert rel(X.cpu().numpy()[rows], (w.V[rows] / w.s) @ w.U.T) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_moore_penrose_4096x3072_refinement_schedule_as_benchmarked(handle):
    """The benchmark's default: FP32-class loops until a step falls below 1,
    X A X in FP32 class, one FP32-class order-2 step, FP64-class order-2 steps
    until a step is below 1e-5, alpha = 1/s_1^2, cleanup finish in FP64 class."""
    w = W.rectangular(4096, 3072, 2304, 1.0, 1e-4, seed=1)
    alpha = 1.0 / w.s[0] ** 2
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp32_refine",
                           variant="stabilized", switch_tol=0.9, finish="clean", check=True)
    assert info["status"] == 0
    assert info["precision"][0] == 3 and info["precision"][-1] == 6 and info["stabilized_loops"] == 1
    rows = np.random.default_rng(0).choice(3072, 32, replace=False)
    assert rel(X.cpu().numpy()[rows], (w.V[rows] / w.s) @ w.U.T) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_complex_moore_penrose_2048x1536_as_benchmarked(handle):
    """Complex rank 1152, s log-spaced in [1e-4, 1] (the complex workload of the
    benchmark, its FP64-class arm: its embedding has the headline's 4096 x 3072
    shape)."""
    w = W.rectangular_complex(2048, 1536, 1152, 1.0, 1e-4, seed=1)
    alpha = 2.0 / (w.s[0] ** 2 + w.s[-1] ** 2)
    X, info = handle.solve_complex(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp64_tc",
                                   variant="stabilized", switch_tol=0.5, finish="clean", check=True)
    assert info["status"] == 0
    rows = np.random.default_rng(0).choice(1536, 32, replace=False)
    assert rel(X.cpu().numpy()[rows], (w.V[rows] / w.s) @ w.U.conj().T) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_complex_moore_penrose_2048x1536_refinement_as_benchmarked(handle):
    """The complex line's default: the refinement schedule with alpha = 1/s_1^2."""
    w = W.rectangular_complex(2048, 1536, 1152, 1.0, 1e-4, seed=1)
    alpha = 1.0 / w.s[0] ** 2
    X, info = handle.solve_complex(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp32_refine",
                                   variant="stabilized", switch_tol=0.9, finish="clean", check=True)
    assert info["status"] == 0
    rows = np.random.default_rng(0).choice(1536, 32, replace=False)
    assert rel(X.cpu().numpy()[rows], (w.V[rows] / w.s) @ w.U.conj().T) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_drazin_2048_as_benchmarked(handle):
    """Index 2 (256 2x2 Jordan blocks), X0 = A^2 / Tr(A^3), order-18 stop,
    finish A^2 X^5 A^2 + one order-2 step."""
    d = W.drazin_index2(2048, 512, seed=2)
    X, info = handle.solve(dev(d.A), kind="drazin", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18",
                           prec="fp64_tc", finish="clean", check=True)
    assert info["status"] == 0
    B = np.zeros((2048, 2048))
    B[:1536, :1536] = np.linalg.inv(d.C)
    rows = np.random.default_rng(0).choice(2048, 32, replace=False)
    ref = d.P[rows] @ B @ np.linalg.inv(d.P)
    assert rel(X.cpu().numpy()[rows], ref) <= 1e-9
    assert max(info["drazin"]) <= 1e-9


def test_drazin_2048_mixed_schedule_as_benchmarked(handle):
    """The Drazin line's loop-schedule arm: FP32-class growth loops, then FP64-class."""
    d = W.drazin_index2(2048, 512, seed=2)
    X, info = handle.solve(dev(d.A), kind="drazin", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18",
                           prec="fp32", finish="clean", check=True)
    assert info["status"] == 0
    assert 3 in info["precision"] and info["precision"][-1] == 4
    B = np.zeros((2048, 2048))
    B[:1536, :1536] = np.linalg.inv(d.C)
    rows = np.random.default_rng(0).choice(2048, 32, replace=False)
    ref = d.P[rows] @ B @ np.linalg.inv(d.P)
    assert rel(X.cpu().numpy()[rows], ref) <= 1e-9
    assert max(info["drazin"]) <= 1e-9


def test_drazin_2048_refinement_schedule_as_benchmarked(handle):
    """The Drazin line's default: FP32-class loops, X A X, FP64-class order-2
    steps, the finish in FP64 class."""
    d = W.drazin_index2(2048, 512, seed=2)
    X, info = handle.solve(dev(d.A), kind="drazin", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18",
                           prec="fp32_refine", finish="clean", check=True)
    assert info["status"] == 0
    assert info["precision"][0] == 3 and info["precision"][-1] == 6
    # one FP32-class step, then a few FP64-class ones (the min(e_j, e_{j-1}^2)
    # rule ends them: the change keeps the nilpotent block's part)
    assert info["precision"].count(5) == 1 and 1 <= info["precision"].count(6) <= 4
    B = np.zeros((2048, 2048))
    B[:1536, :1536] = np.linalg.inv(d.C)
    rows = np.random.default_rng(0).choice(2048, 32, replace=False)
    ref = d.P[rows] @ B @ np.linalg.inv(d.P)
    assert rel(X.cpu().numpy()[rows], ref) <= 1e-9
    assert max(info["drazin"]) <= 1e-9


def test_uneven_batch_4096_as_benchmarked(handle):
    """4096 problems, m ~ U{32..512}, n ~ U{16..m}: one batched call with the
    FP32-finished schedule; 64 sampled instances against their closed forms."""
    import ctypes as C
    from paper_1604_07893_gb300._lib import Desc, Info
    ws = W.uneven_batch_fast(4096, seed=3)
    As = [dev(w.A) for w in ws]
    Xs = [torch.empty(w.A.shape[1], w.A.shape[0], dtype=torch.float64, device="cuda") for w in ws]
    descs = (Desc * len(ws))(*[handle.make_desc(A, X, alpha=1.0 / w.s[0] ** 2, tol=0.25, stop="order18",
                                                prec="bf16_fp32",
                                                finish="clean") for A, X, w in zip(As, Xs, ws)])
    infos = (Info * len(ws))()
    rc = handle._lib.pinv_solve_batched(handle._h, len(ws), descs, C.c_void_p(0), infos)
    torch.cuda.synchronize()
    assert rc == 0 and all(infos[i].status == 0 for i in range(len(ws)))
    for i in np.random.default_rng(0).choice(len(ws), 64, replace=False):
        w = ws[i]
        assert rel(Xs[i].cpu().numpy(), (w.V / w.s) @ w.U.T) <= 1e-4


def test_serving_sizes_256_to_8192(handle):
    """One SPD request of every serving size submitted together (BF16 then
    FP32-class, symmetric products); sampled rows of each result against
    Q diag(1/lambda) Q^T."""
    reqs = []
    for i, n in enumerate([256, 512, 1024, 2048, 4096, 8192]):
        Q, lam = W.spd_fast(n, seed=100 + i)
        Qd = dev(Q)
        A = handle.gemm(Qd * dev(lam), Qd, trans_b=True, prec="fp64_tc")
        A = (0.5 * (A + A.T)).contiguous()
        X = torch.empty(n, n, dtype=torch.float64, device="cuda")
        rid = handle.submit(A, X, G=torch.eye(n, dtype=torch.float64, device="cuda"), kind="outer_g", alpha=1.0,
                            tol=1e-6, prec="bf16_fp32", symmetric=True)
        reqs.append((rid, n, Q, lam, X, A))
    pending = {r[0] for r in reqs}
    status = {}
    while pending:
        for rid in list(pending):
            out = handle.poll(rid)
            if out is not None:
                status[rid] = out[0]
                pending.discard(rid)
    for rid, n, Q, lam, X, _ in reqs:
        assert status[rid] == 0
        rows = np.random.default_rng(n).choice(n, 16, replace=False)
        assert rel(X.cpu().numpy()[rows], (Q[rows] / lam) @ Q.T) <= 1e-4


def test_drazin_index_of_the_2048_workload(handle):
    """ind(A) = 2 for the 2048 workload (256 2x2 Jordan blocks): ranks 2048,
    1792, 1536, 1536."""
    d = W.drazin_index2(2048, 512, seed=2)
    l, ranks = handle.drazin_index(dev(d.A))
    assert l == 2 and ranks == [2048, 1792, 1536, 1536]
