"""pinv_submit / pinv_poll: continuous batching of preconditioner requests
(SPD, G = I, the approximate-inverse family) under an HBM budget."""

import time

import numpy as np
import pytest

from paper_1604_07893_gb300 import workloads as W
from tests.helpers import rel, spd_inverse

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def make_request(n, seed, lam_min=1e-3):
    s = W.spd(n, lam_min, 1.0, seed=seed)
    A, G = dev(s.A), dev(np.eye(n))
    X = torch.empty(n, n, dtype=torch.float64, device="cuda")
    return s, A, G, X


def drain(h, ids, limit_s=120.0):
    """Poll until every request is final (polls return at once; the groups
    advance on the device between them)."""
    done = {}
    t0 = time.time()
    while len(done) < len(ids) and time.time() - t0 < limit_s:
        for i in ids:
            if i not in done:
                r = h.poll(i)
                if r is not None:
                    done[i] = r
    return done


@pytest.mark.parametrize("prec", ["fp64_tc", "mixed_bf16"])
def test_each_result_is_the_same_alone_and_in_the_mix(cuda, prec):
    from paper_1604_07893_gb300 import Handle
    h = Handle(0)
    sizes = [64, 256, 128, 64, 300, 128, 64]
    reqs = [make_request(n, seed=i) for i, n in enumerate(sizes)]
    kw = dict(kind="outer_g", tol=1e-12, prec=prec, symmetric=True)
    ids = []
    for j, (s, A, G, X) in enumerate(reqs):
        ids.append(h.submit(A, X, G=G, alpha=1.0 / s.lam.max(), **kw))
        if j % 3 == 2:                     # later requests arrive while earlier ones run
            h.poll(ids[0])
    done = drain(h, ids)
    assert len(done) == len(ids)
    for (s, A, G, X), i in zip(reqs, ids):
        status, info = done[i]
        assert status == 0
        X1, _ = h.solve(A, G=G, alpha=1.0 / s.lam.max(), **kw)
        assert rel(X.cpu().numpy(), X1.cpu().numpy()) <= 1e-10     # alone vs in the mix
        assert rel(X.cpu().numpy(), spd_inverse(s)) <= 1e-9
        assert info["ms"] > 0
    h.close()


def test_late_arrivals_overlap_with_running_requests(cuda):
    """A slow request (kappa 1e4) admitted first; fast requests (kappa 10)
    submitted after it has started must finish while it is still running."""
    from paper_1604_07893_gb300 import Handle
    h = Handle(0)
    slow = make_request(256, seed=1, lam_min=1e-4)
    sid = h.submit(slow[1], slow[3], G=slow[2], kind="outer_g", alpha=1.0, tol=1e-12, prec="fp64_tc")
    assert h.poll(sid) is None                 # admitted, first loop issued
    fast = [make_request(64, seed=10 + i, lam_min=0.1) for i in range(3)]
    fids = [h.submit(f[1], f[3], G=f[2], kind="outer_g", alpha=1.0, tol=1e-12, prec="fp64_tc")
            for f in fast]
    order = []
    t0 = time.time()
    while len(order) < 4 and time.time() - t0 < 120:
        for i in [sid] + fids:
            if i not in order and h.poll(i) is not None:
                order.append(i)
    assert order[-1] == sid                     # the fast ones overtook it
    assert rel(slow[3].cpu().numpy(), spd_inverse(slow[0])) <= 1e-9
    h.close()


def test_budget_admission_and_rejection(cuda):
    from paper_1604_07893_gb300 import Handle, PinvError
    budget = 64 << 20
    h = Handle(0, hbm_budget_bytes=budget)
    big = make_request(2048, seed=3)
    with pytest.raises(PinvError) as e:
        h.submit(big[1], big[3], G=big[2], kind="outer_g", alpha=1.0, tol=1e-12, prec="fp64_tc")
    assert e.value.code == -2
    reqs = [make_request(256, seed=20 + i) for i in range(6)]
    ids = [h.submit(A, X, G=G, kind="outer_g", alpha=1.0 / s.lam.max(), tol=1e-12, prec="fp64_tc")
           for s, A, G, X in reqs]
    done = drain(h, ids)
    assert len(done) == len(ids)
    for (s, A, G, X), i in zip(reqs, ids):
        assert done[i][0] == 0
        assert rel(X.cpu().numpy(), spd_inverse(s)) <= 1e-9
    h.close()


def test_admission_queue_cap_rejects_and_counts(cuda):
    """max_queued bounds the backlog: submissions beyond it are rejected with
    PINV_ERR_BUSY and counted; admitted requests still complete correctly and
    the counters add up (submitted = completed at the end, none queued)."""
    from paper_1604_07893_gb300 import Handle, PinvError
    h = Handle(0, max_queued=3)
    reqs = [make_request(128, seed=40 + i) for i in range(8)]
    ids, rejected = [], 0
    for s, A, G, X in reqs:
        try:
            ids.append((h.submit(A, X, G=G, kind="outer_g", alpha=1.0 / s.lam.max(), tol=1e-12,
                                 prec="fp64_tc"), s, X))
        except PinvError as e:
            assert e.code == -9
            rejected += 1
    assert len(ids) == 3 and rejected == 5          # nothing polled yet: the queue holds 3
    st = h.serving_stats()
    assert st["queued"] == 3 and st["rejected"] == 5 and st["submitted"] == 3
    done = drain(h, [i for i, _, _ in ids])
    assert len(done) == 3
    for i, s, X in ids:
        assert done[i][0] == 0
        assert rel(X.cpu().numpy(), spd_inverse(s)) <= 1e-9
        assert done[i][1]["tensor_flops"] > 0
    st = h.serving_stats()
    assert st["queued"] == 0 and st["running"] == 0 and st["completed"] == 3 and st["admitted"] == 3
    h.close()
