"""GPU checks of the tcgen05 slice engine (through pinv_gemm / pinv_step /
pinv_solve) against extended-precision references and the oracle.

Error bounds, per element, relative to (|op(A)| |op(B)|)_ij:
* FP64-class (7 exact base-256 slices, 28 products): 4e-16 (native FP64
  rounding is about K u / sqrt(K) ~ 1e-16 here; the slices hold 55 bits and
  the dropped products with s + t = 7 are each at most 2^-56 of the row and
  column maxima);
* FP32-class (4 slices, 10 products): 5e-9 (31 bits; the dropped products
  with s + t = 4 are each at most 2^-32 of the row/column maxima);
* BF16 (one round-to-nearest slice, FP32 accumulation): 2^-7.
"""

import numpy as np
import pytest

from oracle import hyperpower as H
from oracle import precision as PM
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import drazin_closed_form, pinv_closed_form, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOUND = {"fp64_tc": 4e-16, "fp32": 5e-9, "mixed_bf16": 2.0 ** -7}


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


def check_gemm(h, A, B, ta, tb, prec):
    opA = A.T if ta else A
    opB = B.T if tb else B
    ref = opA.astype(np.longdouble) @ opB.astype(np.longdouble)
    scale = np.abs(opA) @ np.abs(opB)
    C = h.gemm(dev(A), dev(B), trans_a=ta, trans_b=tb, prec=prec)
    torch.cuda.synchronize()
    err = (np.abs(C.cpu().numpy() - ref) / np.maximum(scale, 1e-300)).astype(np.float64)
    return float(err.max())


@pytest.mark.parametrize("prec", ["fp64_tc", "fp32", "mixed_bf16"])
@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (1, 1, 1), (200, 136, 300), (130, 70, 2100),
                                   (257, 129, 4101)])
def test_gemm_against_extended_precision(handle, prec, M, N, K):
    rng = np.random.default_rng(M * 31 + N * 7 + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-4, 4, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-4, 4, (1, N)))
    assert check_gemm(handle, A, B, False, False, prec) <= BOUND[prec]


@pytest.mark.parametrize("prec", ["fp64_tc", "fp32"])
@pytest.mark.parametrize("M,N,K", [(2048, 2560, 1100), (2176, 1152, 3000)])
def test_gemm_more_tiles_than_sms_against_extended_precision(handle, prec, M, N, K):
    """Multi-chunk products with more 128 x 128 tiles than SMs, in a number
    that does not divide among them (320 and 153 tiles on 152 SMs): a CTA
    walks several tiles, and the last wave is partial; every sampled row is
    checked against the extended-precision product."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    C = handle.gemm(dev(A), dev(B), prec=prec).cpu().numpy()
    rows = np.unique(np.concatenate([np.arange(0, M, 16), [M - 1]]))
    ref = A[rows].astype(np.longdouble) @ B.astype(np.longdouble)
    scale = np.abs(A[rows]) @ np.abs(B)
    err = (np.abs(C[rows] - ref) / np.maximum(scale, 1e-300)).astype(np.float64)
    assert float(err.max()) <= BOUND[prec]
    # and the deterministic engine: the same product twice is identical
    C2 = handle.gemm(dev(A), dev(B), prec=prec).cpu().numpy()
    assert np.array_equal(C, C2)


@pytest.mark.parametrize("ta,tb", [(True, False), (False, True), (True, True)])
def test_gemm_transposes(handle, ta, tb):
    rng = np.random.default_rng(5)
    M, N, K = 150, 90, 333
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    assert check_gemm(handle, A, B, ta, tb, "fp64_tc") <= BOUND["fp64_tc"]


def test_gemm_fp64_tc_matches_dmma(handle):
    rng = np.random.default_rng(6)
    A = dev(rng.standard_normal((384, 512)))
    B = dev(rng.standard_normal((512, 256)))
    c1 = handle.gemm(A, B, prec="fp64_tc")
    c2 = handle.gemm(A, B, prec="fp64")
    assert float((c1 - c2).abs().max() / c2.abs().max()) < 1e-14


@pytest.mark.parametrize("m,n", [(64, 48), (48, 64), (200, 136), (257, 65)])
def test_one_loop_fp64_tc_matches_naive_step(handle, m, n):
    w = W.rectangular(m, n, None, 1.0, 1e-2, seed=m * 7 + n)
    X = H.x0_moore_penrose(w.A, H.alpha_pan_schreiber(w.s[0], w.s[-1]))
    for _ in range(2):
        ref = H.hyperpower_step(w.A, X, side=H.choose_side(m, n))
        got, _ = handle.step(dev(w.A), dev(X), prec="fp64_tc")
        got = got.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        X = ref


@pytest.mark.parametrize("m,n", [(200, 136), (136, 200)])
def test_one_bf16_loop_matches_the_bf16_model(handle, m, n):
    """One loop with BF16 products (FP32 accumulation; the linear combinations
    formed in FP32 in the final pass), against the CPU model of the same loop
    (oracle/precision.py: the same rounded operands, combinations in FP64)
    and the exact FP64 step.  Ragged tiles on both sides; the iterate is two
    exact loops into the growth phase, so that every term of the loop matters.
    A dropped or mis-signed term moves the result by O(1); the BF16 rounding
    itself moves it by a few per cent at most."""
    w = W.rectangular(m, n, None, 1.0, 1e-2, seed=m + 3 * n)
    side = H.choose_side(m, n)
    X = H.x0_moore_penrose(w.A, 1.0 / w.s[0] ** 2)
    for _ in range(2):
        X = H.hyperpower_step(w.A, X, side=side)
    ref = H.hyperpower_step(w.A, X, side=side)
    model = PM.pm_loop(w.A, X, PM.bf16_product, side)
    got, step = handle.step(dev(w.A), dev(X), prec="mixed_bf16")
    got = got.cpu().numpy()
    e_model = rel(model, ref)
    assert e_model < 0.05
    assert rel(got, model) <= 0.25 * e_model + 1e-4
    assert rel(got, ref) <= 1.5 * e_model + 1e-4
    step_model = float(np.linalg.norm(model - X) / np.linalg.norm(X))
    assert abs(step - step_model) <= 1e-2 * step_model


@pytest.mark.parametrize("variant", ["plain", "stabilized"])
def test_solve_fp64_tc_rank_deficient(handle, variant):
    w = W.rectangular(512, 384, 288, 1.0, 1e-4, seed=1)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                     variant="stabilised" if variant == "stabilized" else "plain", finish="moore_penrose")
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, variant=variant, finish="clean",
                           prec="fp64_tc", check=True)
    assert info["status"] == 0
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


@pytest.mark.parametrize("prec", ["mixed_bf16", "fp32"])
def test_mixed_solve_full_rank(handle, prec):
    """Full column rank (no null block to grow): low-precision early loops are
    corrected by the FP64-class loops that follow."""
    w = W.rectangular(300, 200, None, 1.0, 1e-3, seed=4)
    alpha = 1.0 / w.s[0] ** 2
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-12, prec=prec, finish="clean", check=True)
    assert info["status"] == 0
    assert 1 in info["precision"] or prec == "fp32"
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert rel(X.cpu().numpy(), pinv_closed_form(w)) <= 1e-9


@pytest.mark.parametrize("m,n,r", [(512, 384, 288), (300, 420, 250)])
def test_fp32_class_schedule_on_a_rank_deficient_problem(handle, m, n, r):
    """FP32-class loops while the iterate grows, then FP64-class loops, then the
    finish, with alpha = 1/s_1^2 (kappa 1e4 on the range): the same answer as
    the FP64 oracle to 1e-9, on both residual sides; the precision record shows
    the growth loops in FP32 class and the last loops in FP64 class."""
    w = W.rectangular(m, n, r, 1.0, 1e-4, seed=12)
    alpha = 1.0 / w.s[0] ** 2
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-2, stop=H.STOP_ORDER18, alpha=alpha,
                     finish="moore_penrose")
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp32", variant="stabilized",
                           switch_tol=0.9, finish="clean", check=True)
    assert info["status"] == 0
    prec = info["precision"]
    assert prec[0] == 3 and prec[-1] == 4 and sorted(prec) == prec
    assert info["stabilized_loops"] >= 1
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert rel(X.cpu().numpy(), pinv_closed_form(w)) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


@pytest.mark.parametrize("m,n,r", [(512, 384, 288), (300, 420, 250)])
def test_refinement_schedule_on_a_rank_deficient_problem(handle, m, n, r):
    """FP32-class loops until a step falls below 1, X A X in FP32 class, one
    FP32-class order-2 step, FP64-class order-2 steps until a step is below
    1e-5, then the finish: the same answer as the FP64 oracle to 1e-9 on both
    residual sides; the record shows the FP32-class loops, then the order-2
    steps (codes 5 and 6)."""
    w = W.rectangular(m, n, r, 1.0, 1e-4, seed=12)
    alpha = 1.0 / w.s[0] ** 2
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-2, stop=H.STOP_ORDER18, alpha=alpha,
                     finish="moore_penrose")
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp32_refine",
                           variant="stabilized", switch_tol=0.9, finish="clean", check=True)
    assert info["status"] == 0
    prec = info["precision"]
    loops = [p for p in prec if p == 3]
    steps = [e for p, e in zip(prec, info["history"]) if p in (5, 6)]
    assert prec == loops + [5] + [6] * (len(steps) - 1) and 2 <= len(steps) <= 4
    assert min(steps[-1], steps[-2] ** 2) < 1e-5 and info["stabilized_loops"] == 1
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert rel(X.cpu().numpy(), pinv_closed_form(w)) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_refinement_schedule_needs_the_finish_a_single_solve_and_its_kinds(handle):
    w = W.rectangular(96, 64, 48, 1.0, 1e-2, seed=3)
    _, info = handle.solve(dev(w.A), alpha=1.0, prec="fp32_refine", finish="none", raise_on_error=False)
    assert info["status"] == -1
    _, info = handle.solve(dev(w.A), kind="outer_g", G=dev(np.ascontiguousarray(w.A.T)), alpha=1.0,
                           prec="fp32_refine", finish="clean", raise_on_error=False)
    assert info["status"] == -1
    from paper_1604_07893_gb300._lib import PinvError
    with pytest.raises(PinvError) as e:
        handle.solve_batched([dev(w.A)], alpha=1.0, prec="fp32_refine", finish="clean")
    assert e.value.code == -1


def test_mixed_solve_spd(handle):
    s = W.spd(512, 1e-3, 1.0, seed=5)
    alpha = 1.0 / s.lam.max()          # BF16 loops need alpha <= 1/lambda_max
    X, info = handle.solve(dev(s.A), kind="outer_g", G=dev(np.eye(512)), alpha=alpha, tol=1e-12,
                           prec="mixed_bf16")
    inv = (s.Q / s.lam) @ s.Q.T
    assert info["status"] == 0
    assert rel(X.cpu().numpy(), inv) <= 1e-9


def test_nonfinite_input_reported_on_tensor_cores(handle):
    A = np.ones((40, 30))
    A[3, 7] = np.nan
    X, info = handle.solve(dev(A), alpha=0.01, prec="fp64_tc", raise_on_error=False)
    assert info["status"] == -3


def test_gemm_fp64_tc_wide_dynamic_range(handle):
    """Rows and columns spanning 1e-30 .. 1e30: slices are cut from normalised
    rows and rescaled in the epilogue, so no product leaves the FP32 range."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((96, 200)) * 10.0 ** rng.uniform(-30, 30, (96, 1))
    B = rng.standard_normal((200, 80)) * 10.0 ** rng.uniform(-30, 30, (1, 80))
    assert check_gemm(handle, A, B, False, False, "fp64_tc") <= BOUND["fp64_tc"]


@pytest.mark.parametrize("K", [64, 200, 500, 20000, 70000])
def test_gemm_k_guards(handle, K):
    """Inner dimensions that exercise the engine's accumulation rules: at
    K <= 512 several pairs of a diagonal share one accumulator (g pairs with
    g * K <= 1024); at K = 20000 a diagonal has more than 127 drains of
    1024-deep chunks (the int32 sums are flushed mid-diagonal); at K = 70000
    the exact int64 Horner sum stops one diagonal earlier (|C| must stay below
    2^62) and the rest is added in FP64.  Extremal digits: entries of
    magnitude 1 - 2^-53 have a leading digit 128, so slice products reach
    their bound 2^14."""
    rng = np.random.default_rng(K)
    M, N = 24, 40
    A = rng.choice([-1.0, 1.0], (M, K)) * (1.0 - 2.0 ** -53)
    B = rng.standard_normal((K, N))
    B[:, 0] = 1.0 - 2.0 ** -53   # a column of equal extremal entries: long same-sign runs
    A[0, :] = 1.0 - 2.0 ** -53
    assert check_gemm(handle, A, B, False, False, "fp64_tc") <= BOUND["fp64_tc"]


def test_low_precision_on_rectangular_requires_the_finish(handle):
    """Theorem 6.2: on m != n the block the loop does not contract keeps the
    BF16/FP32 rounding; the library refuses such a schedule without the finish."""
    from paper_1604_07893_gb300 import PinvError
    w = W.rectangular(100, 60, None, 1.0, 1e-2, seed=2)
    for prec in ("mixed_bf16", "fp32"):
        with pytest.raises(PinvError) as e:
            handle.solve(dev(w.A), alpha=1.0, tol=1e-12, prec=prec)
        assert e.value.code == -1


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_symmetric_hint_matches_full_products(handle, prec):
    """A symmetric A with G = I: the symmetric-output products (upper tiles,
    mirrored) give the same inverse as the full products."""
    s = W.spd(300, 1e-3, 1.0, seed=9)
    G = dev(np.eye(300))
    alpha = 1.0 / s.lam.max()
    Xf, i1 = handle.solve(dev(s.A), kind="outer_g", G=G, alpha=alpha, tol=1e-12, prec=prec)
    Xs, i2 = handle.solve(dev(s.A), kind="outer_g", G=G, alpha=alpha, tol=1e-12, prec=prec, symmetric=True)
    assert i1["status"] == 0 and i2["status"] == 0
    assert rel(Xs.cpu().numpy(), Xf.cpu().numpy()) <= 1e-11
    assert rel(Xs.cpu().numpy(), (s.Q / s.lam) @ s.Q.T) <= 1e-9


def test_fp32_finished_schedule(handle):
    """PINV_PREC_BF16_FP32: BF16 growth loops then FP32-class to the end; the
    result carries FP32-class accuracy (u_fp32 kappa) on a nonsingular problem."""
    s = W.spd(400, 1e-3, 1.0, seed=12)
    X, info = handle.solve(dev(s.A), kind="outer_g", G=dev(np.eye(400)), alpha=1.0, tol=1e-12,
                           prec="bf16_fp32", symmetric=True)
    assert info["status"] == 0
    assert set(info["precision"]) <= {1, 3} and info["precision"][-1] == 3
    err = rel(X.cpu().numpy(), (s.Q / s.lam) @ s.Q.T)
    assert err <= 1e-4


def test_order18_stop_parity(handle):
    w = W.rectangular(512, 384, 288, 1.0, 1e-4, seed=1)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    kw = dict(tol=1e-2, alpha=alpha, variant="stabilised", switch_tol=0.5, finish="moore_penrose")
    ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), stop=H.STOP_ORDER18, **kw)
    X, info = handle.solve(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", variant="stabilized",
                           switch_tol=0.5, finish="clean", prec="fp64_tc", check=True)
    assert info["iters"] == oinfo.iters and info["stabilized_loops"] == oinfo.stabilised_loops
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert rel(X.cpu().numpy(), pinv_closed_form(w)) <= 1e-9
    assert max(info["penrose"]) <= 1e-9


def test_autotune_routes_small_products_and_keeps_parity():
    """pinv_autotune measures the DMMA / tensor-core crossover on this device;
    after it a small FP64-class solve (DMMA side of the crossover) and a larger
    one (tensor-core side) both still match the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07893_gb300 import Handle
    h = Handle(0)
    try:
        cross = h.autotune()
        assert cross == 0 or 65 <= cross <= 1025
        for (m, n, r) in [(64, 48, 40), (512, 384, 288)]:
            w = W.rectangular(m, n, r, 1.0, 1e-3, seed=5)
            alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
            ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                             variant="stabilised", finish="moore_penrose")
            X, info = h.solve(dev(w.A), alpha=alpha, tol=1e-12, variant="stabilized", finish="clean",
                              prec="fp64_tc", check=True)
            assert info["status"] == 0
            assert rel(X.cpu().numpy(), ref) <= 1e-9
            assert max(info["penrose"]) <= 1e-9
    finally:
        h.close()


def test_drazin_order18_finish_parity(handle):
    """The Drazin family with the order-18 stop (step < 1e-2) and the finish
    A^l X^{2l+1} A^l + one order-2 step, FP64-class products: same loop count as the
    oracle, result within 1e-9 of the oracle and of the closed form."""
    d = W.drazin_index2(256, 64, seed=2)
    alpha = 1.0 / np.trace(np.linalg.matrix_power(d.A, 3))
    ref, oinfo = H.solve(d.A, H.x0_drazin(d.A, 2, alpha), tol=1e-2, stop=H.STOP_ORDER18, alpha=alpha,
                         finish="drazin", drazin_index=2)
    X, info = handle.solve(dev(d.A), kind="drazin", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18",
                           finish="clean", prec="fp64_tc", check=True)
    assert info["status"] == 0
    assert info["iters"] == oinfo.iters
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert rel(X.cpu().numpy(), drazin_closed_form(d)) <= 1e-9
    assert max(info["drazin"]) <= 1e-9


@pytest.mark.parametrize("n,nil", [(256, 64), (600, 150)])
def test_drazin_fp32_class_schedule_parity(handle, n, nil):
    """The Drazin family in the mixed schedule (FP32-class growth loops, then
    FP64-class loops and the finish in FP64 class): within 1e-9 of the FP64
    oracle and of the closed form, Drazin residuals below 1e-9."""
    d = W.drazin_index2(n, nil, seed=2)
    alpha = 1.0 / np.trace(np.linalg.matrix_power(d.A, 3))
    ref, _ = H.solve(d.A, H.x0_drazin(d.A, 2, alpha), tol=1e-2, stop=H.STOP_ORDER18, alpha=alpha,
                     finish="drazin", drazin_index=2)
    X, info = handle.solve(dev(d.A), kind="drazin", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18",
                           finish="clean", prec="fp32", check=True)
    assert info["status"] == 0
    assert info["precision"][0] == 3 and info["precision"][-1] == 4
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert rel(X.cpu().numpy(), drazin_closed_form(d)) <= 1e-9
    assert max(info["drazin"]) <= 1e-9


@pytest.mark.parametrize("n,nil", [(256, 64), (600, 150)])
def test_drazin_refinement_schedule_parity(handle, n, nil):
    """The Drazin family in the refinement schedule (FP32-class loops, X A X,
    FP64-class order-2 steps, the finish in FP64 class): within 1e-9 of the
    FP64 oracle and of the closed form, Drazin residuals below 1e-9."""
    d = W.drazin_index2(n, nil, seed=2)
    alpha = 1.0 / np.trace(np.linalg.matrix_power(d.A, 3))
    ref, _ = H.solve(d.A, H.x0_drazin(d.A, 2, alpha), tol=1e-2, stop=H.STOP_ORDER18, alpha=alpha,
                     finish="drazin", drazin_index=2)
    X, info = handle.solve(dev(d.A), kind="drazin", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18",
                           finish="clean", prec="fp32_refine", check=True)
    assert info["status"] == 0
    assert info["precision"][0] == 3 and info["precision"][-1] == 6
    assert rel(X.cpu().numpy(), ref) <= 1e-9
    assert rel(X.cpu().numpy(), drazin_closed_form(d)) <= 1e-9
    assert max(info["drazin"]) <= 1e-9
