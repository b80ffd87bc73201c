"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
printed value (Table 1), a closed-form inverse built from the generators'
factors, a library routine on a special case (SVD pseudoinverse, LAPACK
inverse), an exact rational computation, or an invariant the paper proves.
"""

import math

import numpy as np
import pytest

from oracle import hyperpower as H
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import drazin_closed_form, example1, pinv_closed_form, rel, spd_inverse


# --------------------------------------------------------------------------
# coefficients (Section 2)
# --------------------------------------------------------------------------

def test_coefficients_solve_the_printed_systems():
    c = H.coefficients()
    a1, a2, a3, b1, b2, mu, psi = (c[k] for k in ("a1", "a2", "a3", "b1", "b2", "mu", "psi"))
    # the seven equations after Eq. hyper18-33
    eqs = [mu + a1 + b1 - 1,
           a2 + psi + a1 * b1 + b2 - 1,
           2 * a3 + a2 * b1 + a1 * b2 - 1,
           2 + a1 * a3 + a3 * b1 + a2 * b2 - 1,
           a1 + a2 * a3 + b1 + a3 * b2 - 1,
           a2 + a3 ** 2 + b2 - 1,
           2 * a3 - 1]
    assert max(abs(e) for e in eqs) < 1e-14
    # the c-system after Eq. simplify1 and the d-system after Eq. simplify2
    assert abs(c["c1"] + c["c2"] + c["c3"] - a1) < 1e-14
    assert abs(2 + c["c1"] * c["c2"] - a2) < 1e-14
    assert abs(c["c1"] + c["c2"] - a3) < 1e-14
    assert abs(c["d1"] + 0.5 - b1) < 1e-14
    assert abs((8 * c["d2"] + math.sqrt(93) + 3) / 8 - b2) < 1e-14


def test_factorisation_expands_to_all_ones():
    """(1+y)(T(y)S(y) + mu y^2 + psi y^4) = sum_{i<18} y^i as polynomials (Eq. PM
    against Eq. hyper18): multiply the coefficient vectors out."""
    c = H.coefficients()
    P = np.polynomial.polynomial
    L1 = [1, 0, c["c1"], 0, 1]
    L2 = [1, 0, c["c2"], 0, 1]
    M = P.polymul(L1, L2)
    T = P.polyadd(M, [0, 0, c["c3"]])
    S = P.polyadd(M, [0, 0, c["d1"], 0, c["d2"]])
    Z = P.polyadd(P.polymul(T, S), [0, 0, c["mu"], 0, c["psi"]])
    Y = P.polymul([1, 1], Z)
    assert len(Y) == 18
    assert np.max(np.abs(Y - 1.0)) < 1e-13


# --------------------------------------------------------------------------
# the step
# --------------------------------------------------------------------------

@pytest.mark.parametrize("side", ["left", "right"])
def test_factorised_step_equals_naive_step(side):
    w = W.rectangular(64, 48, None, 1.0, 1e-2, seed=0)
    for alpha in (1.0, 0.5):
        X = H.x0_moore_penrose(w.A, alpha)
        for _ in range(3):
            a = H.hyperpower_step(w.A, X, side=side)
            b = H.pm_step(w.A, X, side=side)
            assert rel(b, a) < 1e-13
            X = a


def test_left_and_right_forms_agree():
    w = W.rectangular(40, 24, 18, 1.0, 1e-1, seed=4)
    X = H.x0_moore_penrose(w.A, 1.0)
    for _ in range(2):
        a = H.hyperpower_step(w.A, X, side="left")
        b = H.hyperpower_step(w.A, X, side="right")
        assert rel(a, b) < 1e-13
        X = a


def test_low_orders_are_the_textbook_iterations():
    """p = 2 is Newton-Schulz-Hotelling X(2I - AX) (Eq. schulz) and p = 3 is
    Chebyshev X(3I - AX(3I - AX)) (Eq. chebyshev)."""
    s = W.spd(20, 0.1, 1.0, seed=1)
    A = s.A
    X = 0.7 * np.eye(20)
    I = np.eye(20)
    assert rel(H.hyperpower_step(A, X, p=2), X @ (2 * I - A @ X)) < 1e-14
    assert rel(H.hyperpower_step(A, X, p=3), X @ (3 * I - A @ X @ (3 * I - A @ X))) < 1e-14


def test_residual_powers_invariant():
    """Theorem 3.1: F_{k+1} = F_k^18.  For nonsingular A and X0 commuting with A
    (X0 = alpha I) this is R_{k+1} = R_k^18 exactly."""
    s = W.spd(24, 0.2, 1.0, seed=7)
    X = 1.0 * np.eye(24)
    R0 = H.residual(s.A, X, "right")
    X1 = H.hyperpower_step(s.A, X)
    R1 = H.residual(s.A, X1, "right")
    ref = np.linalg.matrix_power(R0, 18)
    assert np.linalg.norm(R1 - ref) < 1e-13 + 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(R1, 2) < np.linalg.norm(R0, 2) ** 18 * (1 + 1e-6) + 1e-15


# --------------------------------------------------------------------------
# Table 1 (Section 8, Example 1)
# --------------------------------------------------------------------------

def _run_example1(step):
    mpmath = pytest.importorskip("mpmath")
    from fractions import Fraction
    mpmath.mp.dps = 150
    A = np.array([[mpmath.mpf(f.numerator) / f.denominator for f in r] for r in example1("fraction")],
                 dtype=object)
    X = H.x0_drazin(A, 3)
    d = []
    for k in range(30):
        Xn = step(A, X)
        r = H.norm_inf(Xn - X)
        d.append(r)
        X = Xn
        if r <= mpmath.mpf("1e-50"):
            break
    return A, X, k + 1, d


def test_table1_pm_row_reproduced():
    """Table 1, PM column: IT = 5, R_{k+1} = 7.474e-107, rho = 18.00 in
    150-digit arithmetic with X0 = A^3/Tr(A^4) and the infinity-norm stop."""
    A, X, it, d = _run_example1(H.hyperpower_step)
    assert it == 5
    assert float(d[-1]) == pytest.approx(7.474e-107, rel=5e-4)
    assert H.coc([float(x) for x in d])[-1] == pytest.approx(18.0, abs=0.01)


def test_table1_detects_a_planted_mistake():
    """A plausible slip (one term of the hyperpower sum dropped) must break the
    Table 1 pin: the order falls to 17 and the printed residual is missed."""
    A, X, it, d = _run_example1(lambda A, X: H.hyperpower_step(A, X, p=17))
    rho = H.coc([float(x) for x in d])[-1]
    assert abs(rho - 18.0) > 0.5 or float(d[-1]) != pytest.approx(7.474e-107, rel=5e-4)


def test_example1_fp64_matches_exact_drazin_inverse():
    """FP64 oracle against the exact rational A^D = A^3 (A^7)^+ A^3 (sympy)."""
    sp = pytest.importorskip("sympy")
    Af = example1("fraction")
    As = sp.Matrix([[sp.Rational(f.numerator, f.denominator) for f in r] for r in Af])
    AD = As ** 3 * (As ** 7).pinv() * As ** 3
    assert list(AD.row(0)) == [sp.Rational(1, 4), sp.Rational(-1, 4)] + [0] * 10
    assert (As ** 4).trace() == sp.Rational(24592, 625)
    ADf = np.array(AD.tolist(), dtype=float)
    A = example1("float")
    X0 = H.x0_drazin(A, 3)
    X, info = H.solve(A, X0, tol=1e-14, alpha=1.0)
    assert info.status in ("converged", "minimum")
    # FP64 floor for this index-3 matrix: the null block grows 18x per loop
    # from rounding (Theorem 6.2), so the best iterate sits near 2e-12
    assert rel(X, ADf) < 1e-11
    assert H.drazin_residuals(A, X, 3).max() < 1e-11
    assert rel(H.cleanup_drazin(A, X, 3), ADf) < 1e-11


# --------------------------------------------------------------------------
# Moore-Penrose: closed forms and library special cases
# --------------------------------------------------------------------------

def test_mp_64x48_closed_form():
    w = W.rectangular(64, 48, None, 1.0, 1e-2, seed=0)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    X, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    assert info.status == "converged"
    assert rel(X, pinv_closed_form(w)) < 1e-12
    assert H.penrose_residuals(w.A, X).max() < 1e-12
    # the same problem from the rectangular recipe of Section 4
    a2 = H.alpha_rectangular(w.A)
    X2, _ = H.solve(w.A, H.x0_moore_penrose(w.A, a2), tol=1e-12, alpha=a2)
    assert rel(X2, pinv_closed_form(w)) < 1e-12


def test_mp_literal_boundary_alpha_is_wrong():
    """alpha = 2/sigma_max^2 violates the strict condition of Theorem 3.1
    (||F0|| = 1): the top singular direction is annihilated and the iteration
    ends at a different outer inverse.  The oracle must show that failure."""
    w = W.rectangular(64, 48, None, 1.0, 1e-2, seed=0)
    X, _ = H.solve(w.A, H.x0_moore_penrose(w.A, 2.0), tol=1e-12, alpha=2.0)
    assert rel(X, pinv_closed_form(w)) > 1e-6


@pytest.mark.parametrize("m,n,r", [(1, 1, 1), (5, 3, 3), (3, 5, 2), (16, 16, 9), (16, 7, 4), (9, 15, 9)])
def test_mp_tiny_against_svd_pinv(m, n, r):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    ref = np.linalg.pinv(A, rcond=1e-10)
    alpha = H.alpha_rectangular(A)
    X, info = H.solve(A, H.x0_moore_penrose(A, alpha), tol=1e-13, alpha=alpha)
    assert rel(X, ref) < 1e-10
    assert H.penrose_residuals(A, X).max() < 1e-10


def test_mp_rank_deficient_closed_form_and_minimum_stop():
    """Rank-deficient A: the relative step never reaches 1e-16, so the solve
    must end at its minimum (first remark closing Section 6) close to A^+."""
    w = W.rectangular(96, 72, 54, 1.0, 1e-2, seed=11)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    X, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-16, alpha=alpha)
    assert info.status == "minimum"
    assert rel(X, pinv_closed_form(w)) < 1e-11


def test_mp_rank_deficient_kappa_1e4():
    """The 4096 x 3072 family of the headline workload at a reduced size:
    rank 3/4 of n, singular values log-spaced over four decades.  The plain
    loop stalls near 1e-9 (the Penrose symmetry residuals sit there); the
    stabilised variant of Section 7 reaches the closed form to ~1e-12."""
    w = W.rectangular(256, 192, 144, 1.0, 1e-4, seed=12)
    ref = pinv_closed_form(w)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    X, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    assert info.status == "minimum"
    assert rel(X, ref) < 2e-9
    Xs, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                       variant="stabilised")
    assert info.stabilised_loops >= 1
    assert rel(Xs, ref) < 1e-10
    assert H.penrose_residuals(w.A, Xs)[:2].max() < 1e-11


def test_cleanup_then_one_loop_restores_accuracy():
    """The projection alone re-injects rounding of size u*||X||*||A||*||X||; one
    loop after it (which contracts the range block) restores FP64 accuracy and
    brings every Penrose residual well under 1e-9."""
    w = W.rectangular(256, 192, 144, 1.0, 1e-4, seed=12)
    ref = pinv_closed_form(w)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    X, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    assert rel(H.cleanup_moore_penrose(w.A, X), ref) > 1e-11       # the projection alone
    for variant in ("plain", "stabilised"):
        Xf, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                           variant=variant, finish="moore_penrose")
        assert info.finished
        assert rel(Xf, ref) < 1e-11
        assert H.penrose_residuals(w.A, Xf).max() < 3e-10


# --------------------------------------------------------------------------
# Drazin and general outer inverses
# --------------------------------------------------------------------------

def test_drazin_family_closed_form():
    d = W.drazin_index2(40, 10, seed=2)
    X, info = H.solve(d.A, H.x0_drazin(d.A, 2), tol=1e-13, alpha=1.0)
    ref = drazin_closed_form(d)
    assert rel(X, ref) < 1e-11
    assert H.drazin_residuals(d.A, X, 2).max() < 1e-11


def test_outer_inverse_with_prescribed_range_and_null_space():
    """A^(2)_{R(G),N(G)} = G (AG)^# (group inverse of B = AG, B^# = B (B^3)^+ B);
    G = V_s V_s^T A^T has rank s < r so that GA has a real positive spectrum."""
    w = W.rectangular(30, 20, 20, 1.0, 1e-1, seed=5)
    rng = np.random.default_rng(9)
    Vs = np.linalg.qr(rng.standard_normal((20, 6)))[0]
    G = Vs @ Vs.T @ w.A.T
    B = w.A @ G
    ref = G @ (B @ np.linalg.pinv(B @ B @ B, rcond=1e-12) @ B)
    lam = np.linalg.eigvalsh(Vs.T @ w.A.T @ w.A @ Vs)
    alpha = 2.0 / (lam.max() + lam.min())
    X, info = H.solve(w.A, H.x0_general(G, alpha), tol=1e-13, alpha=alpha)
    assert rel(X, ref) < 1e-11
    assert rel(X @ w.A @ X, X) < 1e-11                      # Eq. 1: X in A{2}
    assert np.linalg.matrix_rank(X, 1e-8) == 6


def test_spd_inverse_closed_form_and_lapack():
    s = W.spd(64, 1e-3, 1.0, seed=5)
    alpha = 2.0 / (s.lam.max() + s.lam.min())
    X, info = H.solve(s.A, alpha * np.eye(64), tol=1e-13, alpha=alpha)
    assert rel(X, spd_inverse(s)) < 1e-11
    assert rel(X, np.linalg.solve(s.A, np.eye(64))) < 1e-11


# --------------------------------------------------------------------------
# stabilised step and cleanup: the block analysis of Theorems 6.2 and 7.1
# --------------------------------------------------------------------------

def _blocks(w, X):
    """SVD blocks of Theorem 6.2: X = V_full [[X11, X12], [X21, X22]] U_full^T."""
    m, n = w.A.shape
    r = len(w.s)
    Uf = np.linalg.svd(w.U, full_matrices=True)[0]  # columns: U then its complement
    Vf = np.linalg.svd(w.V, full_matrices=True)[0]
    Uf[:, :r] = w.U
    Vf[:, :r] = w.V
    B = Vf.T @ X @ Uf
    return B[:r, :r], B[:r, r:], B[r:, :r], B[r:, r:]


def test_plain_step_multiplies_null_block_by_18_and_stabilised_step_removes_it():
    w = W.rectangular(24, 16, 10, 1.0, 0.5, seed=3)
    rng = np.random.default_rng(0)
    Aplus = pinv_closed_form(w)
    E = 1e-7 * rng.standard_normal(Aplus.shape)
    X = Aplus + E
    b0 = _blocks(w, X)
    plain = _blocks(w, H.hyperpower_step(w.A, X))
    stab = _blocks(w, H.stabilised_step(w.A, X))
    # Theorem 6.2: E22 -> 18 E22, E12 and E21 unchanged, E11 removed (first order)
    assert np.linalg.norm(plain[3] - 18 * b0[3]) < 1e-3 * np.linalg.norm(b0[3])
    assert np.linalg.norm(plain[1] - b0[1]) < 1e-3 * np.linalg.norm(b0[1])
    assert np.linalg.norm(plain[2] - b0[2]) < 1e-3 * np.linalg.norm(b0[2])
    assert np.linalg.norm(plain[0] - np.diag(1 / w.s)) < 1e-3 * np.linalg.norm(b0[0] - np.diag(1 / w.s))
    # Theorem 7.1: the extra X A X removes E22 to first order
    assert np.linalg.norm(stab[3]) < 1e-3 * np.linalg.norm(b0[3])


def test_cleanup_fixes_the_pseudoinverse_and_removes_off_blocks():
    w = W.rectangular(24, 16, 10, 1.0, 0.5, seed=3)
    Aplus = pinv_closed_form(w)
    assert rel(H.cleanup_moore_penrose(w.A, Aplus), Aplus) < 1e-14
    rng = np.random.default_rng(1)
    X = Aplus + 1e-7 * rng.standard_normal(Aplus.shape)
    b = _blocks(w, H.cleanup_moore_penrose(w.A, X))
    b0 = _blocks(w, X)
    for i in (1, 2, 3):
        assert np.linalg.norm(b[i]) < 1e-3 * np.linalg.norm(b0[i])


def test_drazin_cleanup_fixes_the_drazin_inverse():
    d = W.drazin_index2(20, 6, seed=8)
    AD = drazin_closed_form(d)
    assert rel(H.cleanup_drazin(d.A, AD, 2), AD) < 1e-12


def test_stabilised_solve_converges_and_switches():
    w = W.rectangular(96, 72, 54, 1.0, 1e-2, seed=11)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    X, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-14, alpha=alpha,
                      variant="stabilised", switch_tol=1e-3)
    assert info.stabilised_loops >= 1
    assert rel(X, pinv_closed_form(w)) < 1e-11


# --------------------------------------------------------------------------
# initial values, scaling, stop measures, residual functions
# --------------------------------------------------------------------------

def test_alpha_recipes_by_hand():
    A = np.array([[1.0, -2.0], [3.0, 4.0]])
    # ||A||_1 = max column sum = 6, ||A||_inf = max row sum = 7
    assert H.alpha_rectangular(A) == pytest.approx(1.0 / 42.0)
    assert H.alpha_pan_schreiber(1.0, 1e-2) == pytest.approx(2.0 / 1.0001)


def test_paper_stop_measure_by_hand():
    X = np.zeros((2, 2))
    Xn = np.array([[3.0, 0.0], [0.0, 4.0]])
    # ||Xn - X||_F = 5; 18^2 * 0.5 = 162
    assert H.stop_measure(Xn, X, 2, 0.5, H.STOP_PAPER) == pytest.approx(5.0 / 162.0)


def test_residual_functions_see_wrong_answers():
    w = W.rectangular(20, 12, None, 1.0, 0.1, seed=2)
    Aplus = pinv_closed_form(w)
    assert H.penrose_residuals(w.A, Aplus).max() < 1e-13
    bad = Aplus.copy()
    bad[0, 0] += 1e-3
    assert H.penrose_residuals(w.A, bad).max() > 1e-6
    d = W.drazin_index2(16, 4, seed=1)
    AD = drazin_closed_form(d)
    assert H.drazin_residuals(d.A, AD, 2).max() < 1e-12
    assert H.drazin_residuals(d.A, AD + 1e-4, 2).max() > 1e-6


def test_nonfinite_input_stops():
    A = np.ones((4, 3))
    A[0, 0] = np.nan
    X, info = H.solve(A, H.x0_moore_penrose(A, 0.1), alpha=0.1)
    assert info.status == "nonfinite"


def test_order18_stop_reaches_the_same_accuracy_in_fewer_loops():
    """Theorem 3.1 (F_{k+1} = F_k^18): after a loop whose step is below 1e-2 the
    iterate is at the rounding floor, so stopping there loses nothing."""
    w = W.rectangular(256, 192, 144, 1.0, 1e-4, seed=12)
    ref = pinv_closed_form(w)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    Xa, ia = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                     variant="stabilised", finish="moore_penrose")
    Xb, ib = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-2, stop=H.STOP_ORDER18, alpha=alpha,
                     variant="stabilised", switch_tol=0.5, finish="moore_penrose")
    assert ib.loops_run < ia.loops_run and ib.stabilised_loops >= 1
    assert rel(Xb, ref) < 3e-12 and rel(Xa, ref) < 3e-12
    assert H.penrose_residuals(w.A, Xb).max() < 3e-10


def test_drazin_normal_initial_value_for_any_spectrum():
    """Eigenvalues all around the annulus 0.5 <= |z| <= 2: Tr(A^3) is not a
    usable scaling for A^2, but G = A^l (A^{2l+1})^T A^l (same range and null
    space as A^D) converges to the closed-form Drazin inverse."""
    d = W.drazin_index2(96, 24, seed=2, sector=np.pi)
    X, info = H.solve(d.A, H.x0_drazin_normal(d.A, 2), tol=1e-2, stop=H.STOP_ORDER18, alpha=1.0)
    assert info.status == "converged"
    assert rel(X, drazin_closed_form(d)) < 1e-10
    assert H.drazin_residuals(d.A, X, 2).max() < 1e-10


# --------------------------------------------------------------------------
# degenerate inputs (closed forms)
# --------------------------------------------------------------------------

def test_zero_matrix_is_a_fixed_point():
    """A = 0: X0 = alpha A^T = 0 is already A^dagger = 0; the first loop leaves
    it unchanged and the solve stops there (a zero step measures 0)."""
    A = np.zeros((6, 4))
    X, info = H.solve(A, H.x0_moore_penrose(A, 1.0), tol=1e-12, alpha=1.0)
    assert info.status == "converged" and info.iters == 1
    assert np.array_equal(X, np.zeros((4, 6)))


def test_rank_one_closed_form():
    """A = u v^T has A^dagger = v u^T / (|u|^2 |v|^2)."""
    rng = np.random.default_rng(7)
    u, v = rng.standard_normal(9), rng.standard_normal(5)
    A = np.outer(u, v)
    exact = np.outer(v, u) / (u @ u) / (v @ v)
    alpha = 1.0 / ((u @ u) * (v @ v))          # 1 / sigma_1^2
    X, info = H.solve(A, H.x0_moore_penrose(A, alpha), tol=1e-12, alpha=alpha)
    assert info.status in ("converged", "minimum")
    assert rel(X, exact) < 1e-13


@pytest.mark.parametrize("A,exact", [(np.eye(5), np.eye(5)), (np.array([[-4.0]]), np.array([[-0.25]])),
                                     (np.diag([2.0, 0.5, 0.0]), np.diag([0.5, 2.0, 0.0]))])
def test_identity_scalar_and_diagonal(A, exact):
    """Inverses with obvious closed forms: I, a 1 x 1 matrix, a singular diagonal."""
    alpha = 1.0 / (H.norm_inf(A) * H.norm_inf(A.T))
    X, info = H.solve(A, H.x0_moore_penrose(A, alpha), tol=1e-12, alpha=alpha)
    assert info.status in ("converged", "minimum")
    assert rel(X, exact) < 1e-13


# --------------------------------------------------------------------------
# the index of a matrix (Section 4)
# --------------------------------------------------------------------------

def test_drazin_index_of_example1_is_the_printed_3():
    """Section 8, Example 1 states l = ind(A) = 3 for the printed matrix."""
    l, ranks = H.drazin_index(example1())
    assert l == 3
    assert ranks[3] == ranks[4] < ranks[2]


@pytest.mark.parametrize("case,expected", [("nonsingular", 0), ("diagonal_singular", 1), ("jordan4", 4),
                                           ("family", 2)])
def test_drazin_index_by_construction(case, expected):
    """Index 0 for a nonsingular matrix, 1 for a singular diagonalizable one,
    k for a nilpotent Jordan block of size k, 2 for the generator's family
    (2 x 2 Jordan blocks)."""
    rng = np.random.default_rng(3)
    if case == "nonsingular":
        A = rng.standard_normal((6, 6)) + 6 * np.eye(6)
    elif case == "diagonal_singular":
        Q = np.linalg.qr(rng.standard_normal((5, 5)))[0]
        A = Q @ np.diag([2.0, -1.0, 0.5, 0.0, 0.0]) @ Q.T
    elif case == "jordan4":
        A = np.diag(np.ones(3), 1)
    else:
        A = W.drazin_index2(64, 16, seed=2).A
    l, ranks = H.drazin_index(A)
    assert l == expected
    assert ranks[l] == ranks[l + 1] and (l == 0 or ranks[l - 1] > ranks[l])


# --------------------------------------------------------------------------
# complex matrices (Section 1.1: the method is stated over C, A^* the
# conjugate transpose; Theorem 3.1 holds as stated)
# --------------------------------------------------------------------------

def test_complex_norm_and_conjugate_transpose_by_hand():
    x = np.array([[3 + 4j, 0], [1j, -1]])
    assert H.fro(x) == pytest.approx(math.sqrt(25 + 1 + 1))
    assert np.array_equal(H.ct(x), np.array([[3 - 4j, -1j], [0, -1]]))
    assert np.array_equal(H.x0_moore_penrose(x, 2.0), 2.0 * np.array([[3 - 4j, -1j], [0, -1]]))


def test_complex_mp_closed_form_and_lapack():
    w = W.rectangular_complex(40, 28, None, 1.0, 1e-2, seed=21)
    ref = pinv_closed_form(w)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    X, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    assert info.status == "converged" and X.dtype == np.complex128
    assert rel(X, ref) < 1e-12
    assert rel(X, np.linalg.pinv(w.A)) < 1e-12
    assert H.penrose_residuals(w.A, X).max() < 1e-12
    # the rectangular recipe of Section 4 with complex moduli
    a2 = H.alpha_rectangular(w.A)
    assert a2 == pytest.approx(1.0 / (np.abs(w.A).sum(axis=0).max() * np.abs(w.A).sum(axis=1).max()))
    X2, _ = H.solve(w.A, H.x0_moore_penrose(w.A, a2), tol=1e-12, alpha=a2)
    assert rel(X2, ref) < 1e-12
    # a plausible slip: X0 = alpha A^T without the conjugate has the wrong range
    with np.errstate(over="ignore", invalid="ignore"):
        Xt, _ = H.solve(w.A, alpha * w.A.T, tol=1e-12, alpha=alpha, max_iter=30)
    assert not rel(Xt, ref) < 1e-3
    # and the Penrose residual function sees a conjugation slip in X
    assert H.penrose_residuals(w.A, ref.conj())[0] > 1e-2


def test_complex_mp_rank_deficient_with_finish():
    w = W.rectangular_complex(72, 54, 40, 1.0, 1e-3, seed=22)
    ref = pinv_closed_form(w)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    for variant in ("plain", "stabilised"):
        X, info = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                          variant=variant, finish="moore_penrose")
        assert info.finished
        assert rel(X, ref) < 1e-11
        assert H.penrose_residuals(w.A, X).max() < 1e-10


def test_complex_solve_of_a_real_matrix_is_the_real_solve():
    w = W.rectangular(30, 20, None, 1.0, 1e-2, seed=3)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    Xr, ir = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    Ac = w.A.astype(np.complex128)
    Xc, ic = H.solve(Ac, H.x0_moore_penrose(Ac, alpha), tol=1e-12, alpha=alpha)
    assert ic.iters == ir.iters
    assert np.abs(Xc.imag).max() == 0.0
    assert rel(Xc.real, Xr) < 1e-14


def test_complex_residual_powers_invariant():
    """R_{k+1} = R_k^18 (Theorem 3.1, right form) for a Hermitian positive
    definite A from X0 = alpha I."""
    s = W.hpd_complex(24, 0.1, 1.0, seed=7)
    alpha = 2.0 / 1.1
    I = np.eye(24, dtype=np.complex128)
    X1 = H.hyperpower_step(s.A, alpha * I)
    R0, R1 = I - alpha * s.A, I - s.A @ X1
    assert rel(R1, np.linalg.matrix_power(R0, 18)) < 1e-12


def test_complex_inverse_from_identity_g():
    s = W.hpd_complex(48, 1e-2, 1.0, seed=8)
    alpha = 2.0 / (1.0 + 1e-2)
    X, info = H.solve(s.A, H.x0_general(np.eye(48, dtype=np.complex128), alpha), tol=1e-13, alpha=alpha)
    assert rel(X, spd_inverse(s)) < 1e-12
    assert rel(X, np.linalg.inv(s.A)) < 1e-12


def test_complex_drazin_closed_form():
    d = W.drazin_complex(40, 10, seed=23)
    ref = drazin_closed_form(d)
    l, ranks = H.drazin_index(d.A)
    assert l == 2 and ranks[:4] == [40, 35, 30, 30]
    # Section 4's trace scaling, alpha = 1/Tr(A^3) complex as it stands
    X, info = H.solve(d.A, H.x0_drazin(d.A, 2), tol=1e-13, alpha=1.0)
    assert rel(X, ref) < 1e-11
    assert H.drazin_residuals(d.A, X, 2).max() < 1e-11
    # a real scaling 1/Re Tr(A^3)
    tr = H.trace(H.matpow(d.A, 3))
    X2, _ = H.solve(d.A, H.x0_drazin(d.A, 2, 1.0 / tr.real), tol=1e-13, alpha=1.0)
    assert rel(X2, ref) < 1e-11
    # G = A^l (A^{2l+1})^* A^l converges for a spectrum all around the annulus
    d2 = W.drazin_complex(48, 12, seed=24, sector=np.pi)
    X3, info3 = H.solve(d2.A, H.x0_drazin_normal(d2.A, 2), tol=1e-2, stop=H.STOP_ORDER18, alpha=1.0)
    assert info3.status == "converged"
    assert rel(X3, drazin_closed_form(d2)) < 1e-10


# --------------------------------------------------------------------------
# approximate-inverse preconditioner (Section 8, Example 3)
# --------------------------------------------------------------------------

def test_jacobi_initial_value_by_hand():
    A = np.array([[2.0, 1.0], [3.0, -4.0]])
    assert np.array_equal(H.x0_jacobi(A), np.array([[0.5, 0.0], [0.0, -0.25]]))
    Z = np.array([[1 + 1j, 0], [2, 2j]])
    assert np.allclose(H.x0_jacobi(Z), np.diag([0.5 - 0.5j, -0.5j]), rtol=0, atol=1e-16)
    with pytest.raises(ValueError):
        H.x0_jacobi(np.array([[0.0, 1.0], [1.0, 1.0]]))


def test_chop_by_hand():
    x = np.array([[1e-6, -2e-5, 3.0], [-1e-7, 0.0, 1e-5]])
    assert np.array_equal(H.chop(x, 1e-5), np.array([[0.0, -2e-5, 3.0], [0.0, 0.0, 1e-5]]))
    z = np.array([1.0 + 1e-6j, 1e-6 + 2j, 1e-7 - 1e-7j])
    assert np.array_equal(H.chop(z, 1e-5), np.array([1.0 + 0j, 2j, 0j]))


def test_jacobi_of_a_diagonal_matrix_is_its_inverse():
    A = np.diag([2.0, -3.0, 0.5, 7.0])
    X, steps = H.preconditioner(A, loops=1)
    assert rel(X, np.linalg.inv(A)) < 1e-15


@pytest.mark.parametrize("complex_", [False, True])
def test_one_loop_preconditioner_residual_is_the_18th_power(complex_):
    """X1 from X0 = D^{-1}: I - X1 A = (I - X0 A)^18 and I - A X1 = (I - A X0)^18
    (X0 (I - A X0)^j = (I - X0 A)^j X0), so ||I - X1 A|| = ||R0^18||."""
    A = W.grid_operator(6, seed=7, complex_=complex_)
    n = A.shape[0]
    I = np.eye(n)
    X0 = H.x0_jacobi(A)
    X1, steps = H.preconditioner(A, loops=1)
    L0 = I - X0 @ A
    assert rel(I - X1 @ A, np.linalg.matrix_power(L0, 18)) < 1e-12
    assert rel(I - A @ X1, np.linalg.matrix_power(I - A @ X0, 18)) < 1e-12
    rho = max(abs(np.linalg.eigvals(L0)))
    assert rho < 0.95
    assert max(abs(np.linalg.eigvals(I - X1 @ A))) == pytest.approx(rho ** 18, rel=1e-6)
    # a second loop: the 18^2 = 324th power
    X2, _ = H.preconditioner(A, loops=2)
    assert np.linalg.norm(I - X2 @ A) < 10 * np.linalg.norm(np.linalg.matrix_power(L0, 324)) + 1e-13


def test_chopped_preconditioner_stays_close_and_sparse():
    A = W.grid_operator(8, seed=8)
    X1, _ = H.preconditioner(A, loops=1)
    Xc, _ = H.preconditioner(A, loops=1, chop_eps=1e-5)
    assert np.count_nonzero(Xc) < np.count_nonzero(X1)
    diff = Xc - X1
    assert np.abs(diff.real).max() < 1e-5 and np.abs(diff.imag).max() < 1e-5
    assert np.array_equal(Xc, H.chop(X1, 1e-5))


# --------------------------------------------------------------------------
# outer inverses through G (Section 1.1): weighted Moore-Penrose, Bott-Duffin;
# the alpha of a general G
# --------------------------------------------------------------------------

def _sqrtm_spd(s, power):
    return (s.Q * s.lam ** power) @ s.Q.conj().T


@pytest.mark.parametrize("complex_", [False, True])
def test_weighted_moore_penrose_through_g(complex_):
    """A^+_{MN} = A^(2)_{R(N^{-1}A^*M), N(N^{-1}A^*M)}: X0 = alpha N^{-1} A^* M.
    Pinned to the closed form N^{-1/2} (M^{1/2} A N^{-1/2})^+ M^{1/2} and to the
    four weighted Penrose equations AXA = A, XAX = X, (MAX)^* = MAX, (NXA)^* = NXA."""
    if complex_:
        w = W.rectangular_complex(30, 20, 14, 1.0, 1e-2, seed=31)
        Ms, Ns = W.hpd_complex(30, 0.2, 5.0, seed=32), W.hpd_complex(20, 0.5, 2.0, seed=33)
    else:
        w = W.rectangular(30, 20, 14, 1.0, 1e-2, seed=31)
        Ms, Ns = W.spd(30, 0.2, 5.0, seed=32), W.spd(20, 0.5, 2.0, seed=33)
    A, M, N = w.A, Ms.A, Ns.A
    G = _sqrtm_spd(Ns, -1.0) @ H.ct(A) @ M
    a = H.alpha_general(A, G)
    X, info = H.solve(A, H.x0_general(G, a), tol=1e-13, alpha=a, finish=None)
    ref = (_sqrtm_spd(Ns, -0.5) @ np.linalg.pinv(_sqrtm_spd(Ms, 0.5) @ A @ _sqrtm_spd(Ns, -0.5), rcond=1e-10)
           @ _sqrtm_spd(Ms, 0.5))
    assert rel(X, ref) < 1e-10
    assert rel(A @ X @ A, A) < 1e-10 and rel(X @ A @ X, X) < 1e-10
    MAX, NXA = M @ A @ X, N @ X @ A
    assert rel(H.ct(MAX), MAX) < 1e-10 and rel(H.ct(NXA), NXA) < 1e-10
    # and it is not the plain pseudoinverse
    assert rel(ref, np.linalg.pinv(A)) > 1e-3


def test_bott_duffin_inverse_through_g():
    """A^{(-1)}_{(L)} = P_L (A P_L + P_{L^perp})^{-1} = A^(2)_{L, L^perp} for A
    positive definite: X0 = alpha P_L."""
    s = W.spd(40, 0.05, 1.0, seed=34)
    P, Q = W.subspace_projector(40, 25, seed=35)
    a = H.alpha_general(s.A, P)
    X, info = H.solve(s.A, H.x0_general(P, a), tol=1e-13, alpha=a)
    ref = P @ np.linalg.inv(s.A @ P + (np.eye(40) - P))
    assert rel(X, ref) < 1e-11
    assert rel(P @ X, X) < 1e-11 and rel(X @ P, X) < 1e-11
    # on L it inverts the compression Q^T A Q
    assert rel(Q.T @ X @ Q, np.linalg.inv(Q.T @ s.A @ Q)) < 1e-11


def test_general_alpha_bounds_the_spectrum_of_ga():
    w = W.rectangular(50, 30, None, 1.0, 1e-2, seed=36)
    for A, G in ((w.A, w.A.T), (w.A.T.copy(), w.A.copy()), (W.spd(30, 1e-3, 1.0, seed=37).A, np.eye(30))):
        a = H.alpha_general(A, G)
        lam = np.linalg.eigvals(G @ A)
        assert a * np.abs(lam).max() <= 1.0 + 1e-12
        assert a * np.abs(lam).max() > 0.1   # not needlessly small on these families


@pytest.mark.parametrize("m,n", [(300, 200), (200, 300)])
def test_outer_finish_keeps_a_weighted_inverse_and_sharpens_it(m, n):
    """Rank-deficient weighted Moore-Penrose: the plain loop ends near 1e-9
    (Theorem 6.2's persistent blocks); X A X removes them (1e-12), while the
    Moore-Penrose projection (XA)^T X (AX)^T would land far from A^+_{MN}."""
    w = W.rectangular(m, n, 150, 1.0, 1e-3, seed=31)
    Ms, Ns = W.spd(m, 0.2, 5.0, seed=32), W.spd(n, 0.5, 2.0, seed=33)
    A = w.A
    G = _sqrtm_spd(Ns, -1.0) @ A.T @ Ms.A
    ref = (_sqrtm_spd(Ns, -0.5) @ np.linalg.pinv(_sqrtm_spd(Ms, 0.5) @ A @ _sqrtm_spd(Ns, -0.5), rcond=1e-10)
           @ _sqrtm_spd(Ms, 0.5))
    a = H.alpha_general(A, G)
    X, _ = H.solve(A, H.x0_general(G, a), tol=1e-12, alpha=a)
    Xf, info = H.solve(A, H.x0_general(G, a), tol=1e-12, alpha=a, finish="outer")
    assert info.finished
    assert rel(X, ref) > 1e-10 and rel(Xf, ref) < 3e-12
    assert rel(H.cleanup_moore_penrose(A, X), ref) > 0.1
