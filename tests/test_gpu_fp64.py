"""GPU parity of the FP64 path against the oracle (through the C ABI).

Tolerances (FP64 products on both sides):
* one loop: the factorised seven-product step against the naive 17-product
  oracle step -- both exact up to rounding, relative Frobenius difference and
  per-element difference <= 1e-12 of the largest entry;
* whole solves: relative Frobenius difference <= 1e-9 (the FP64-finished bar
  at kappa <= 1e4) and <= 1e-12 where the oracle itself reaches 1e-14.
"""

import math

import numpy as np
import pytest

from oracle import hyperpower as H
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import drazin_closed_form, example1, pinv_closed_form, rel

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


# -------------------------------------------------------------------------- products

@pytest.mark.parametrize("M,N,K", [(48, 48, 64), (200, 136, 300), (256, 200, 96), (512, 512, 64),
                                   (520, 300, 100), (2048, 2048, 64), (7, 5, 3)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, True)])
def test_dmma_tiles_against_extended_precision(handle, M, N, K, ta, tb):
    """The FP64 kernel picks an 8 (K split over the warps), 16, 32 or 64 CTA
    tile by the grid it would fill (these shapes reach all four on a 152-SM
    part); every tile keeps the FP64 bound |C - AB| <= K u (|A| |B|)
    elementwise."""
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    ref = opA.astype(np.longdouble) @ opB.astype(np.longdouble)
    C = host(handle.gemm(dev(A), dev(B), trans_a=ta, trans_b=tb, prec="fp64"))
    err = (np.abs(C - ref) / (np.abs(opA) @ np.abs(opB))).astype(np.float64).max()
    assert err <= K * 2.0 ** -53


# -------------------------------------------------------------------------- one loop

@pytest.mark.parametrize("m,n", [(64, 48), (48, 64), (1, 1), (200, 136), (136, 200), (130, 130),
                                 (17, 129), (257, 65)])
def test_one_pm_loop_matches_naive_order18_step(handle, m, n):
    w = W.rectangular(m, n, None, 1.0, 1e-2, seed=m * 7 + n)
    A = w.A
    X = H.x0_moore_penrose(A, H.alpha_pan_schreiber(w.s[0], w.s[-1]))
    for _ in range(2):
        ref = H.hyperpower_step(A, X, side=H.choose_side(m, n))
        got, step = handle.step(dev(A), dev(X))
        assert_close(host(got), ref, 1e-12)
        assert step == pytest.approx(float(np.linalg.norm(ref - X) / np.linalg.norm(X)), rel=1e-10)
        X = ref


@pytest.mark.parametrize("m,n", [(96, 72), (72, 96)])
def test_one_stabilised_loop_matches_oracle(handle, m, n):
    w = W.rectangular(m, n, 54, 1.0, 1e-1, seed=3)
    X = H.x0_moore_penrose(w.A, 1.0)
    for _ in range(3):
        X = H.hyperpower_step(w.A, X)
    ref = H.stabilised_step(w.A, X, side=H.choose_side(m, n))
    got, _ = handle.step(dev(w.A), dev(X), stabilized=True)
    assert_close(host(got), ref, 1e-12)


# -------------------------------------------------------------------------- solves

def test_solve_64x48_matches_oracle_and_closed_form(handle):
    """The small Moore-Penrose case: 64 x 48, s log-spaced in [1e-2, 1]."""
    w = W.rectangular(64, 48, None, 1.0, 1e-2, seed=0)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, check=True)
    assert info["status"] == 0 and info["iters"] == oinfo.iters
    assert_close(host(X), ref, 1e-12)
    assert rel(host(X), pinv_closed_form(w)) < 1e-12
    assert max(info["penrose"]) < 1e-12


def test_solve_literal_boundary_alpha_fails_like_the_oracle(handle):
    """alpha = 2/s_max^2 (the edge of Theorem 3.1's condition) reaches another
    outer inverse on both sides."""
    w = W.rectangular(64, 48, None, 1.0, 1e-2, seed=0)
    X, info = handle.solve(dev(w.A), alpha=2.0, tol=1e-12)
    assert rel(host(X), pinv_closed_form(w)) > 1e-6


@pytest.mark.parametrize("variant", ["plain", "stabilized"])
def test_solve_rank_deficient_kappa_1e4(handle, variant):
    """Reduced form of the 4096 x 3072 rank-2304 workload (rank 3n/4,
    s log-spaced in [1e-4, 1]), with the cleanup-and-one-loop finish."""
    w = W.rectangular(512, 384, 288, 1.0, 1e-4, seed=1)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                     variant="stabilised" if variant == "stabilized" else "plain",
                     finish="moore_penrose")
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, variant=variant, finish="clean",
                           check=True)
    assert info["status"] == 0
    assert rel(host(X), ref) <= 1e-9
    assert rel(host(X), pinv_closed_form(w)) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_solve_wide_matrix_right_side(handle):
    w = W.rectangular(70, 150, 60, 1.0, 1e-2, seed=9)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-13, alpha=alpha, finish="moore_penrose")
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-13, finish="clean")
    assert info["side"] == "right"
    assert rel(host(X), ref) < 1e-11


def test_solve_drazin_family(handle):
    d = W.drazin_index2(256, 64, seed=2)
    ref, _ = H.solve(d.A, H.x0_drazin(d.A, 2), tol=1e-13, alpha=1.0)
    X, info = handle.solve(dev(d.A), kind="drazin", drazin_index=2, tol=1e-13, check=True)
    assert info["status"] == 0
    assert rel(host(X), ref) < 1e-10
    assert rel(host(X), drazin_closed_form(d)) < 1e-10
    assert max(info["drazin"]) < 1e-10
    tr = np.trace(np.linalg.matrix_power(d.A, 3))
    assert info["alpha"] == pytest.approx(1.0 / tr, rel=1e-12)


def test_solve_example1_drazin(handle):
    """Section 8, Example 1 in FP64: the printed index-3 matrix."""
    A = example1()
    ref, _ = H.solve(A, H.x0_drazin(A, 3), tol=1e-14, alpha=1.0)
    X, info = handle.solve(dev(A), kind="drazin", drazin_index=3, tol=1e-14)
    assert rel(host(X), ref) < 1e-10
    assert abs(host(X)[0, 0] - 0.25) < 1e-10 and abs(host(X)[0, 1] + 0.25) < 1e-10


def test_solve_outer_inverse_with_G(handle):
    w = W.rectangular(30, 20, 20, 1.0, 1e-1, seed=5)
    rng = np.random.default_rng(9)
    Vs = np.linalg.qr(rng.standard_normal((20, 6)))[0]
    G = np.ascontiguousarray(Vs @ Vs.T @ w.A.T)
    lam = np.linalg.eigvalsh(Vs.T @ w.A.T @ w.A @ Vs)
    alpha = 2.0 / (lam.max() + lam.min())
    ref, _ = H.solve(w.A, H.x0_general(G, alpha), tol=1e-13, alpha=alpha)
    X, info = handle.solve(dev(w.A), kind="outer_g", G=dev(G), alpha=alpha, tol=1e-13)
    assert rel(host(X), ref) < 1e-11


def test_solve_spd_nonsingular(handle):
    s = W.spd(300, 1e-3, 1.0, seed=5)
    alpha = 2.0 / (s.lam.max() + s.lam.min())
    ref, _ = H.solve(s.A, H.x0_general(np.eye(300), alpha), tol=1e-13, alpha=alpha)
    X, info = handle.solve(dev(s.A), kind="outer_g", G=dev(np.eye(300)), alpha=alpha, tol=1e-13)
    assert rel(host(X), ref) < 1e-11


def test_paper_stop_rule(handle):
    """Eq. stopreliable with the Frobenius norm (Section 8, Example 2) on a
    Hilbert matrix H_{100x90}, X0 = 2/(s1^2 + sr^2) H^T."""
    A = W.hilbert(100, 90)
    s = np.linalg.svd(A, compute_uv=False)
    s_r = s[s > 1e-15 * s[0]][-1]          # numerically nonzero: sigma_r of Section 4
    alpha = 2.0 / (s[0] ** 2 + s_r ** 2)
    ref, oinfo = H.solve(A, H.x0_moore_penrose(A, alpha), tol=1e-5, stop=H.STOP_PAPER, alpha=alpha)
    X, info = handle.solve(dev(A), alpha=alpha, tol=1e-5, stop="paper")
    assert info["iters"] == oinfo.iters
    assert rel(host(X), ref) < 1e-6


def test_alpha_estimate(handle):
    w = W.rectangular(123, 77, None, 2.0, 1e-2, seed=4)
    assert handle.alpha_estimate(dev(w.A)) == pytest.approx(H.alpha_rectangular(w.A), rel=1e-12)
    X, info = handle.solve(dev(w.A), alpha=0.0, tol=1e-12)
    assert info["alpha"] == pytest.approx(H.alpha_rectangular(w.A), rel=1e-12)


def test_host_buffers_equal_device_buffers(handle):
    w = W.rectangular(100, 60, None, 1.0, 1e-2, seed=6)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    Xd, _ = handle.solve(dev(w.A), alpha=alpha, tol=1e-12)
    Xh, info = handle.solve(np.ascontiguousarray(w.A), alpha=alpha, tol=1e-12, host=True)
    assert info["status"] == 0
    assert np.array_equal(Xh, host(Xd))


def test_deterministic(handle):
    w = W.rectangular(200, 150, 120, 1.0, 1e-3, seed=8)
    a = handle.solve(dev(w.A), alpha=1.0, tol=1e-12)[0]
    b = handle.solve(dev(w.A), alpha=1.0, tol=1e-12)[0]
    assert torch.equal(a, b)


def test_batched_equals_single(handle):
    ws = W.uneven_batch(6, seed=3, m_hi=200)
    As = [dev(w.A) for w in ws]
    Xs, infos = handle.solve_batched(As, alpha=0.0, tol=1e-12)
    for A, X, info in zip(As, Xs, infos):
        X1, _ = handle.solve(A, alpha=0.0, tol=1e-12)
        # the batch pads each problem to a multiple of 64: same iterate, other rounding
        assert rel(host(X), host(X1)) <= 1e-11


def test_submit_poll_equals_solve(handle):
    ws = [W.rectangular(80 + 10 * i, 50, None, 1.0, 1e-2, seed=i) for i in range(3)]
    As = [dev(w.A) for w in ws]
    Xs = [torch.empty(50, A.shape[0], dtype=torch.float64, device="cuda") for A in As]
    ids = [handle.submit(A, X, alpha=0.0, tol=1e-12) for A, X in zip(As, Xs)]
    done = {}
    import time
    t0 = time.time()
    while len(done) < len(ids) and time.time() - t0 < 120:   # polls return at once; GPU work is async
        for i in ids:
            if i not in done:
                r = handle.poll(i)
                if r is not None:
                    done[i] = r
    assert len(done) == len(ids)
    for A, X, i in zip(As, Xs, ids):
        assert done[i][0] == 0
        X1, _ = handle.solve(A, alpha=0.0, tol=1e-12)
        assert rel(host(X), host(X1)) <= 1e-11


# -------------------------------------------------------------------------- errors

def test_argument_errors(handle):
    from paper_1604_07893_gb300 import PinvError
    A = dev(np.ones((4, 3)))
    with pytest.raises(PinvError) as e:
        handle.solve(A, kind="drazin", drazin_index=1)      # Drazin needs a square A
    assert e.value.code == -1
    with pytest.raises(PinvError) as e:
        handle.solve(A, alpha=-1.0)
    assert e.value.code == -1
    with pytest.raises(PinvError) as e:
        handle.solve(dev(np.eye(3)), kind="drazin", drazin_index=0)
    assert e.value.code == -1


def test_nonfinite_input_reported(handle):
    A = np.ones((6, 4))
    A[2, 1] = np.nan
    X, info = handle.solve(dev(A), alpha=0.1, raise_on_error=False)
    assert info["status"] == -3


def test_budget_error():
    from paper_1604_07893_gb300 import Handle, PinvError
    h = Handle(0, hbm_budget_bytes=1 << 20)
    A = dev(np.ones((512, 512)))
    with pytest.raises(PinvError) as e:
        h.solve(A, alpha=1e-3)
    assert e.value.code == -2
    h.close()


# -------------------------------------------------------------------------- full size

@pytest.mark.slow
def test_full_size_rank_deficient_sampled_rows(handle):
    """The 4096 x 3072 rank-2304 workload in FP64, as timed by the benchmark:
    sampled rows of X against the closed form V diag(1/s) U^T, and the
    Penrose residuals computed on the device."""
    w = W.rectangular(4096, 3072, 2304, 1.0, 1e-4, seed=1)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, variant="stabilized", finish="clean",
                           check=True)
    assert info["status"] == 0
    Xh = host(X)
    rows = np.random.default_rng(0).choice(3072, 24, replace=False)
    ref_rows = (w.V[rows] / w.s) @ w.U.T
    assert rel(Xh[rows], ref_rows) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_drazin_normal_on_the_full_annulus(handle, prec):
    """Eigenvalues all around the annulus (where X0 = A^2/Tr(A^3) cannot
    converge): G = A^l (A^{2l+1})^T A^l reaches the closed-form A^D."""
    d = W.drazin_index2(256, 64, seed=2, sector=np.pi)
    ref, oinfo = H.solve(d.A, H.x0_drazin_normal(d.A, 2), tol=1e-2, stop=H.STOP_ORDER18, alpha=1.0,
                         finish="drazin", drazin_index=2)
    X, info = handle.solve(dev(d.A), kind="drazin_normal", drazin_index=2, alpha=0.0, tol=1e-2,
                           stop="order18", finish="clean", prec=prec, check=True)
    assert info["status"] == 0
    assert rel(host(X), drazin_closed_form(d)) < 1e-9
    assert rel(host(X), ref) < 1e-9
    assert max(info["drazin"]) < 1e-9


# -------------------------------------------------------------------------- degenerate inputs

@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_zero_matrix(handle, prec):
    """A = 0: X = A^dagger = 0 exactly, found in one loop like the oracle."""
    A = np.zeros((6, 4))
    ref, oinfo = H.solve(A, H.x0_moore_penrose(A, 1.0), tol=1e-12, alpha=1.0)
    X, info = handle.solve(dev(A), alpha=1.0, tol=1e-12, prec=prec)
    assert info["status"] == 0 and info["iters"] == oinfo.iters == 1
    assert np.array_equal(host(X), ref)
    # the alpha = 0 recipe is undefined for A = 0; any alpha gives X0 = 0, so the
    # solve takes alpha = 1 (as a batched group does) and returns X = 0
    X0, info0 = handle.solve(dev(A), alpha=0.0, tol=1e-12, prec=prec)
    assert info0["status"] == 0 and info0["alpha"] == 1.0 and not host(X0).any()
    G = np.zeros((4, 6))
    Xg, infog = handle.solve(dev(A), kind="outer_g", G=dev(G), alpha=0.0, tol=1e-12, prec=prec)
    assert infog["status"] == 0 and not host(Xg).any()


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("case", ["rank_one", "identity", "scalar", "singular_diagonal"])
def test_degenerate_closed_forms(handle, prec, case):
    rng = np.random.default_rng(7)
    if case == "rank_one":
        u, v = rng.standard_normal(9), rng.standard_normal(5)
        A, exact = np.outer(u, v), np.outer(v, u) / (u @ u) / (v @ v)
    elif case == "identity":
        A, exact = np.eye(5), np.eye(5)
    elif case == "scalar":
        A, exact = np.array([[-4.0]]), np.array([[-0.25]])
    else:
        A, exact = np.diag([2.0, 0.5, 0.0]), np.diag([0.5, 2.0, 0.0])
    alpha = 1.0 / (H.norm_inf(A) * H.norm_inf(A.T))
    ref, _ = H.solve(A, H.x0_moore_penrose(A, alpha), tol=1e-12, alpha=alpha)
    X, info = handle.solve(dev(A), alpha=alpha, tol=1e-12, prec=prec)
    assert info["status"] == 0
    assert rel(host(X), ref) < 1e-12
    assert rel(host(X), exact) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_replayed_loops_serve_new_matrices_of_the_same_shape(handle, prec):
    """Small solves replay their loop from a graph cached in the handle; the
    matrix is copied into the workspace first, so solving a different matrix
    of the same shape (and shapes in between) reuses the graph correctly."""
    cases = [W.rectangular(64, 48, None, 1.0, 1e-2, seed=s) for s in (0, 1)]
    other = W.rectangular(40, 72, None, 1.0, 1e-2, seed=3)
    for w in (cases[0], other, cases[1], cases[0]):
        alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
        ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
        X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, prec=prec)
        assert info["status"] == 0 and info["iters"] == oinfo.iters
        assert rel(host(X), ref) < 1e-12
        assert rel(host(X), pinv_closed_form(w)) < 1e-12


@pytest.mark.parametrize("case", ["example1", "family", "nonsingular", "diagonal_singular", "jordan4"])
def test_drazin_index_matches_the_oracle(handle, case):
    """pinv_drazin_index (ranks from this library's own pseudoinverses) gives
    the oracle's ind(A) and rank sequence (SVD ranks)."""
    rng = np.random.default_rng(3)
    if case == "example1":
        A = example1()
    elif case == "family":
        A = W.drazin_index2(256, 64, seed=2).A
    elif case == "nonsingular":
        A = rng.standard_normal((6, 6)) + 6 * np.eye(6)
    elif case == "diagonal_singular":
        Q = np.linalg.qr(rng.standard_normal((5, 5)))[0]
        A = Q @ np.diag([2.0, -1.0, 0.5, 0.0, 0.0]) @ Q.T
    else:
        A = np.diag(np.ones(3), 1)
    l_ref, ranks_ref = H.drazin_index(A)
    l, ranks = handle.drazin_index(dev(A))
    assert l == l_ref
    assert ranks == ranks_ref


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_device_loop_decisions_match_the_oracle(handle, prec):
    """Small plain solves apply the stop rule on the device: the per-loop stop
    measures, the loop count and the max_iter outcome agree with the oracle."""
    w = W.rectangular(64, 48, None, 1.0, 1e-2, seed=0)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, prec=prec)
    assert info["status"] == 0 and info["iters"] == oinfo.iters and info["loops_run"] == oinfo.loops_run
    for got, want in zip(info["history"][:info["loops_run"]], oinfo.history):
        if want > 1e-9:
            assert abs(got - want) <= 1e-6 * want
    # max_iter: two loops, then PINV_ERR_MAXITER with the second iterate
    ref2, oinfo2 = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha, max_iter=2)
    X2, info2 = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, prec=prec, max_iter=2, raise_on_error=False)
    assert oinfo2.status == "maxiter" and info2["status"] == -5 and info2["iters"] == 2
    assert rel(host(X2), ref2) < 1e-12


@pytest.mark.parametrize("m,n", [(64, 48), (48, 64), (128, 128), (100, 37), (1, 1)])
def test_small_device_loop_solves_match_the_oracle(handle, m, n):
    """Small plain FP64 solves of several shapes (both residual sides, ragged
    tiles, 1 x 1) run their loop on the device: loop count, per-loop measures
    and the result agree with the oracle, and a later solve of another matrix of
    the same shape reuses the cached loop correctly."""
    w = W.rectangular(m, n, None, 1.0, 1e-2, seed=3 * m + n)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, prec="fp64")
    assert info["status"] == 0 and info["iters"] == oinfo.iters and info["loops_run"] == oinfo.loops_run
    for got, want in zip(info["history"][:info["loops_run"]], oinfo.history):
        if want > 1e-9:
            assert abs(got - want) <= 1e-6 * want
    assert rel(host(X), ref) < 1e-12
    w2 = W.rectangular(m, n, None, 1.0, 1e-1, seed=3 * m + n + 1)
    a2 = H.alpha_pan_schreiber(w2.s[0], w2.s[-1])
    ref2, _ = H.solve(w2.A, H.x0_moore_penrose(w2.A, a2), tol=1e-12, alpha=a2)
    X2, _ = handle.solve(dev(w2.A), alpha=a2, tol=1e-12, prec="fp64")
    assert rel(host(X2), ref2) < 1e-12
