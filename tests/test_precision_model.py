"""CPU pins of the product-class model (oracle/precision.py) and the precision
schedules it justifies.

The model's formats are pinned to their definitions (hand cases, torch's own
BF16 conversion, exact rational products); the schedule tests then show, on
the rank-deficient family of the headline workload at 512 x 384 (rank 288,
singular values log-spaced in [1e-4, 1]), which product classes the
iteration tolerates in its early loops:

* FP32-class loops while the iterate grows, one FP64-class loop, then the
  finish (projection + order-2 step), with alpha = 1/sigma_1^2: the result is
  within 3e-12 of the closed-form A^+ -- the same as every loop in FP64
  class.
* The same schedule with alpha = 2/(sigma_1^2 + sigma_r^2) fails: the top
  residual eigenvalue sits at about -1 and the rounding pushes it past.
* BF16 loops at the start fail even with alpha = 1/sigma_1^2: their rounding
  lands in the null block, which grows by 18 per loop (Theorem 6.2) faster
  than the finish can remove it.
* The refinement schedule: the same FP32-class loops up to the first step
  below 1, X A X in FP32 class, one FP32-class order-2 step, then FP64-class
  order-2 steps until min(step, previous step^2) < 1e-5 (one here), then the
  finish: within 3e-12 of A^+ as well.  Without the X A X the second order-2
  step measures the doubled null-block rounding (~1e-4), not the squared
  range error.
* On a full-rank problem (no null block) BF16 growth loops are harmless.
* On the Drazin family (index 2: a nilpotent block, on which I - AX keeps the
  eigenvalue 1), FP32-class growth loops then FP64 class meet the FP64
  accuracy, while one FP8 (per-tensor scaled E4M3) or BF16 first loop already
  makes the iteration fail.
"""

from fractions import Fraction

import numpy as np
import pytest

from oracle import hyperpower as H
from oracle import precision as PM
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import drazin_closed_form, pinv_closed_form, rel


# ----------------------------------------------------------------- formats

def test_round_bits_hand_cases():
    # 1 + 2^-8 is halfway between the BF16 neighbours 1 and 1 + 2^-7: even -> 1
    assert PM.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: even -> 1 + 2^-6
    assert PM.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    # just above the halfway point rounds up
    assert PM.bf16(np.array([1 + 2.0 ** -8 + 2.0 ** -30]))[0] == 1 + 2.0 ** -7
    assert PM.bf16(np.array([-3.0]))[0] == -3.0
    assert PM.bf16(np.array([0.0]))[0] == 0.0
    assert PM.fp32(np.array([1 + 2.0 ** -24]))[0] == 1.0
    assert PM.fp32(np.array([1 + 2.0 ** -23]))[0] == 1 + 2.0 ** -23


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(20000) * np.exp2(np.random.default_rng(1).integers(-20, 20, 20000))
    x32 = x.astype(np.float32).astype(np.float64)      # exactly representable in FP32
    want = torch.from_numpy(x32).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(PM.bf16(x32), want)


def test_e4m3_hand_cases():
    assert PM.e4m3(np.array([448.0, 500.0, -1e9]))[0] == 448.0
    assert PM.e4m3(np.array([500.0]))[0] == 448.0 and PM.e4m3(np.array([-1e9]))[0] == -448.0
    # normal spacing: 4 significant bits; 1.0625 is halfway between 1 and 1.125 -> 1
    assert PM.e4m3(np.array([1.0625]))[0] == 1.0
    assert PM.e4m3(np.array([1.1875]))[0] == 1.25
    # subnormals: multiples of 2^-9; 2^-10 is a tie between 0 and 2^-9 -> 0
    assert PM.e4m3(np.array([2.0 ** -9]))[0] == 2.0 ** -9
    assert PM.e4m3(np.array([2.0 ** -10]))[0] == 0.0
    assert PM.e4m3(np.array([3 * 2.0 ** -10]))[0] == 2 * 2.0 ** -9


# ------------------------------------------------------------ slice product

@pytest.mark.parametrize("S", [1, 2, 4, 7])
def test_digits_are_balanced_and_reconstruct_the_fixed_point_integer(S):
    rng = np.random.default_rng(S)
    X = rng.standard_normal((9, 13)) * np.exp2(rng.integers(-30, 30, (9, 1)))
    X[3, :] = 0.0
    q, e = PM.digits(X, S, axis=1)
    T = 8 * S - 1
    U = np.floor(np.abs(X) * np.exp2(T - e) + 0.5).astype(np.int64)
    total = sum(q[s].astype(np.int64) << (8 * (S - 1 - s)) for s in range(S))
    assert np.array_equal(total, np.where(X < 0, -U, U))
    for s in range(S):
        assert np.all(np.abs(q[s]) <= 128)
    # the line exponent puts the largest entry in [1/2, 1) after scaling
    mx = np.max(np.abs(X), axis=1)
    nz = mx > 0
    assert np.all(mx[nz] * np.exp2(-e[nz, 0]) >= 0.5) and np.all(mx[nz] * np.exp2(-e[nz, 0]) < 1.0)


def _exact_product(A, B):
    Af = [[Fraction(float(v)) for v in row] for row in A]
    Bf = [[Fraction(float(v)) for v in row] for row in B]
    return [[sum(Af[i][k] * Bf[k][j] for k in range(len(Bf))) for j in range(len(Bf[0]))]
            for i in range(len(Af))]


@pytest.mark.parametrize("S,L,bits", [(7, 6, 55), (4, 3, 31)])
def test_slice_product_within_its_truncation_bound(S, L, bits):
    """|C - AB|_ij <= c K 2^-bits rowmax_i colmax_j against the exact rational
    product: the rounding of each operand to T = 8S - 1 bits plus the dropped
    pairs s + t > L (each below 2^(-8(L+1)) of the leading pair)."""
    rng = np.random.default_rng(bits)
    A = rng.standard_normal((6, 40)) * np.exp2(rng.integers(-8, 8, (6, 1)))
    B = rng.standard_normal((40, 5)) * np.exp2(rng.integers(-8, 8, (1, 5)))
    C = PM.slice_product(A, B, S, L)
    E = _exact_product(A, B)
    K = A.shape[1]
    ra = np.max(np.abs(A), axis=1)
    cb = np.max(np.abs(B), axis=0)
    for i in range(A.shape[0]):
        for j in range(B.shape[1]):
            err = abs(Fraction(float(C[i, j])) - E[i][j])
            assert float(err) <= 4 * K * 2.0 ** -bits * ra[i] * cb[j]
    if S == 7:   # FP64 class: as good as a correctly rounded FP64 product here
        assert np.max(np.abs(C - A @ B) / (np.abs(A) @ np.abs(B))) < 1e-14


def test_bf16_product_is_the_product_of_rounded_operands():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((8, 16))
    B = rng.standard_normal((16, 8))
    C = PM.bf16_product(A, B)
    assert np.allclose(C, PM.bf16(A) @ PM.bf16(B), rtol=2 ** -22, atol=0)
    assert np.max(np.abs(C - A @ B)) > 1e-4   # it is not the FP64 product


def test_model_loop_equals_the_naive_step_in_fp64():
    """With exact FP64 products the model's loop (the GPU grouping) equals the
    oracle's naive order-18 step to rounding."""
    w = W.rectangular(40, 30, None, 1.0, 1e-2, seed=4)
    X = H.x0_moore_penrose(w.A, 1.0 / w.s[0] ** 2)
    for side in ("left", "right"):
        got = PM.pm_loop(w.A, X, PM.CLASSES["fp64"], side)
        want = H.hyperpower_step(w.A, X, side=side)
        assert rel(got, want) < 1e-13


def test_order2_step_squares_the_residual():
    """Eq. hyper with p = 2: X' = X + X R (R = I - AX) gives I - AX' = R^2
    exactly in exact arithmetic (left side: I - X'A = (I - XA)^2)."""
    w = W.rectangular(40, 30, None, 1.0, 1e-1, seed=6)
    X = H.x0_moore_penrose(w.A, 1.0 / w.s[0] ** 2)
    R = np.eye(40) - w.A @ X
    Xr = PM.order2_step(w.A, X, PM.CLASSES["fp64"], "right")
    assert np.abs((np.eye(40) - w.A @ Xr) - R @ R).max() < 1e-14
    L = np.eye(30) - X @ w.A
    Xl = PM.order2_step(w.A, X, PM.CLASSES["fp64"], "left")
    assert np.abs((np.eye(30) - Xl @ w.A) - L @ L).max() < 1e-14


# ---------------------------------------------------------------- schedules

@pytest.fixture(scope="module")
def rank_deficient():
    return W.rectangular(512, 384, 288, 1.0, 1e-4, seed=12)


def _schedule(w, alpha, classes, finish="order2"):
    X, steps = PM.run_schedule(w.A, H.x0_moore_penrose(w.A, alpha), classes, finish=finish)
    if not np.all(np.isfinite(X)):
        return np.inf, np.inf, steps
    return rel(X, pinv_closed_form(w)), float(max(H.penrose_residuals(w.A, X))), steps


def test_fp32_class_growth_loops_then_fp64_class_meet_the_fp64_accuracy(rank_deficient):
    w = rank_deficient
    alpha = 1.0 / w.s[0] ** 2
    err, pen, steps = _schedule(w, alpha, ["fp32_class"] * 7 + ["fp64_class"])
    ref_err, ref_pen, ref_steps = _schedule(w, alpha, ["fp64_class"] * 8)
    assert err <= 3e-12 and pen <= 1e-9
    assert ref_err <= 3e-12
    # the growth phase (steps above 1) and the loop count are those of FP64 class
    assert [s > 1 for s in steps] == [s > 1 for s in ref_steps]
    assert steps[6] < 1.0 and steps[7] < 1e-2


def _refine(w, alpha, with_xax=True):
    """FP32-class loops while the step is >= 1 (the loop that first steps below
    1 included), X A X in FP32 class, one FP32-class order-2 step, FP64-class
    order-2 steps until min(step, previous step^2) < 1e-5 (at most 8), the
    finish in FP64 class."""
    A = w.A
    side = H.choose_side(*A.shape)
    f32, f64 = PM.CLASSES["fp32_class"], PM.CLASSES["fp64_class"]
    X = H.x0_moore_penrose(A, alpha)
    loops = []
    for _ in range(20):
        Xn = PM.pm_loop(A, X, f32, side)
        loops.append(float(np.linalg.norm(Xn - X) / np.linalg.norm(X)))
        X = Xn
        if loops[-1] < 1.0:
            break
    if with_xax:
        X = PM.xax(A, X, f32, side)
    steps = []
    for j in range(8):
        Xn = PM.order2_step(A, X, f32 if j == 0 else f64, side)
        steps.append(float(np.linalg.norm(Xn - X) / np.linalg.norm(X)))
        X = Xn
        if j > 0 and min(steps[-1], steps[-2] ** 2) < 1e-5:
            break
    X = PM.finish_moore_penrose(A, X, f64, side, "order2")
    return rel(X, pinv_closed_form(w)), float(max(H.penrose_residuals(A, X))), loops, steps


def test_refinement_schedule_meets_the_fp64_accuracy(rank_deficient):
    w = rank_deficient
    err, pen, loops, steps = _refine(w, 1.0 / w.s[0] ** 2)
    assert len(loops) == 7 and loops[-1] < 1.0 <= loops[-2]
    # two order-2 steps: the first (FP32 class) measures the loop's error
    # (~1e-3), the second (FP64 class) its square
    assert len(steps) == 2 and 1e-4 < steps[0] < 1e-2 and steps[1] < 1e-5
    assert err <= 3e-12 and pen <= 1e-9


def test_refinement_schedule_on_the_right_residual_side():
    """A wide rank-deficient problem (m < n: the right residual I - AX) under
    the same refinement schedule: within 3e-12 of A^+."""
    w = W.rectangular(300, 420, 250, 1.0, 1e-4, seed=12)
    err, pen, loops, steps = _refine(w, 1.0 / w.s[0] ** 2)
    assert H.choose_side(300, 420) == "right"
    assert loops[-1] < 1.0 and len(steps) == 2
    assert err <= 3e-12 and pen <= 1e-9


def test_refinement_without_the_stabilising_product_sees_the_doubled_block(rank_deficient):
    """Without X A X the order-2 steps double the FP32-class rounding outside
    the range (order p multiplies that block by p, Theorem 6.2), so the second
    step's change stays near the first's instead of falling to its square; the
    square of the first step's change is what bounds the range error then."""
    w = rank_deficient
    _, _, _, steps = _refine(w, 1.0 / w.s[0] ** 2, with_xax=False)
    assert steps[1] > 1e-4


@pytest.mark.parametrize("m,n,seed", [(256, 192, 21), (200, 64, 7)])
def test_order18_stop_threshold_of_the_fp32_finished_schedule(m, n, seed):
    """BF16 growth loops, FP32-class loops stopped by the order-18 rule, the
    FP32-class projection and order-18 loop: delta = 0.25 (0.25^18 = 1.5e-11,
    below the FP32 class's 2^-31) keeps the first FP32-class loop whose step is
    below it, one loop before delta = 1e-2, at the same accuracy."""
    w = W.rectangular(m, n, None, 1.0, 1e-3, seed=seed, spacing="loguniform")
    A = w.A
    side = H.choose_side(m, n)
    f32 = PM.CLASSES["fp32_class"]
    out = {}
    for delta in (1e-2, 0.25):
        X = H.x0_moore_penrose(A, 1.0 / w.s[0] ** 2)
        cls, loops = "bf16", 0
        for _ in range(30):
            Xn = PM.pm_loop(A, X, PM.CLASSES[cls], side)
            step = float(np.linalg.norm(Xn - X) / np.linalg.norm(X))
            X, loops = Xn, loops + 1
            if cls == "bf16":
                if step <= 0.5:
                    cls = "fp32_class"
            elif step < delta:
                break
        X = PM.finish_moore_penrose(A, X, f32, side, "order18")
        out[delta] = (loops, rel(X, pinv_closed_form(w)))
    assert out[0.25][0] == out[1e-2][0] - 1
    assert out[0.25][1] <= 1e-6 and out[0.25][1] <= 2 * out[1e-2][1]


def test_fp32_class_loops_fail_with_the_two_sided_alpha(rank_deficient):
    w = rank_deficient
    alpha = 2.0 / (w.s[0] ** 2 + w.s[-1] ** 2)
    err, _, _ = _schedule(w, alpha, ["fp32_class"] * 7 + ["fp64_class"])
    assert err > 1e-3
    # in FP64 class the same alpha is fine: the failure is the rounding at r ~ -1
    ok, _, _ = _schedule(w, alpha, ["fp64_class"] * 8)
    assert ok <= 3e-12


def test_bf16_loops_fail_on_a_rank_deficient_problem(rank_deficient):
    w = rank_deficient
    err, _, _ = _schedule(w, 1.0 / w.s[0] ** 2, ["bf16"] * 2 + ["fp32_class"] * 5 + ["fp64_class"])
    assert err > 1e-3


def test_bf16_growth_loops_are_harmless_without_a_null_block():
    w = W.rectangular(256, 192, None, 1.0, 1e-3, seed=21)
    alpha = 1.0 / w.s[0] ** 2
    classes = ["bf16"] * 4 + ["fp32_class"] + ["fp64_class"] * 2
    X, steps = PM.run_schedule(w.A, H.x0_moore_penrose(w.A, alpha), classes, finish="order18")
    assert rel(X, pinv_closed_form(w)) <= 1e-12


@pytest.fixture(scope="module")
def drazin_family():
    return W.drazin_index2(128, 32, seed=2)


def _drazin_schedule(d, classes):
    X, steps = PM.run_schedule(d.A, H.x0_drazin(d.A, 2), classes, drazin_index=2)
    if not np.all(np.isfinite(X)):
        return np.inf, steps
    return rel(X, drazin_closed_form(d)), steps


def test_drazin_refinement_schedule(drazin_family):
    """FP32-class loops to the first step below 1, X A X, one FP32-class and
    then FP64-class order-2 steps until min(step, previous step^2) < 1e-5, the
    Drazin finish: the FP64 accuracy of the loop schedule."""
    d = drazin_family
    A = d.A
    f32, f64 = PM.CLASSES["fp32_class"], PM.CLASSES["fp64_class"]
    X = H.x0_drazin(A, 2)
    for _ in range(20):
        Xn = PM.pm_loop(A, X, f32, "right")
        step = float(np.linalg.norm(Xn - X) / np.linalg.norm(X))
        X = Xn
        if step < 1.0:
            break
    X = PM.xax(A, X, f32, "right")
    steps = []
    for j in range(8):
        Xn = PM.order2_step(A, X, f32 if j == 0 else f64, "right")
        steps.append(float(np.linalg.norm(Xn - X) / np.linalg.norm(X)))
        X = Xn
        if j > 0 and min(steps[-1], steps[-2] ** 2) < 1e-5:
            break
    X = PM.finish_drazin(A, X, 2, f64)
    ref, _ = _drazin_schedule(d, ["fp64_class"] * 5)
    assert len(steps) <= 4
    assert rel(X, drazin_closed_form(d)) <= max(1e-13, 2 * ref)


def test_drazin_fp32_class_growth_loops_then_fp64_class(drazin_family):
    err, steps = _drazin_schedule(drazin_family, ["fp32_class"] * 3 + ["fp64_class"] * 2)
    ref, _ = _drazin_schedule(drazin_family, ["fp64_class"] * 5)
    assert ref <= 1e-13
    assert err <= 1e-13
    assert steps[-1] < 1e-2   # the order-18 stop fires on the second FP64-class loop


@pytest.mark.parametrize("first", ["fp8", "bf16"])
def test_drazin_low_precision_first_loop_fails(drazin_family, first):
    """After the loop that should have converged, the step grows again (the
    first loop's rounding in the nilpotent block, amplified 18 per loop) and the
    result misses the 1e-9 bar (FP8: it diverges)."""
    err, steps = _drazin_schedule(drazin_family, [first] + ["fp32_class"] * 2 + ["fp64_class"] * 3)
    assert steps[-1] > 1.0
    assert not err <= 1e-9
