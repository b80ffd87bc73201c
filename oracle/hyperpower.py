"""Plain, slow, FP64 CPU oracle for the order-18 hyperpower iteration.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, the package's smoke check and the benchmark's CPU-baseline leg call
it.  It shares no code with the CUDA path: the only thing both sides consume is
the seeded matrices from the input generator module.

What it computes (Pan, Soleymani, Zhao, "Highly efficient computation of
generalized inverse of a matrix"):

* the outer inverse X = A^(2)_{R(G),N(G)} (Section 1.1, Eq. 1 and the
  lemma after it) reached from X0 = alpha*G (Section 2);
* each loop forms the order-18 hyperpower step the obvious way,
  X_{k+1} = X_k (I + R_k + R_k^2 + ... + R_k^17), R_k = I - A X_k
  (Eq. hyper18), with 17 successive products -- NOT the factorised seven-product
  step, which the CUDA path uses and which this module only contains so that a
  test can show the two agree (Eq. PM, Section 2);
* the stabilised loop appends X <- X A X (Eq. PM-modified, Section 7), switched
  on once the step size falls below a threshold (the switching recipe closing
  Section 7);
* stopping by the relative Frobenius step, or by the criterion of Eq.
  stopreliable (Section 4), and stopping once a step in the converged regime
  is no longer a convergent step (the first remark closing Section 6: the
  iteration is not self-correcting for generalized inverses);
* initial values of Section 4: alpha*A^T, A^l/Tr(A^{l+1}), alpha*G, with
  alpha = 2/(sigma_1^2 + sigma_r^2) or 1/(||A||_1 ||A||_inf);
* the approximate-inverse preconditioner of Section 8, Example 3: loops of
  the step from the Jacobi X0 = diag(1/a_ii), each followed by a chop;
* residual checks: the Penrose equations and the Drazin equations;
* the computational order of convergence of Eq. COC (Section 8).

Readings where the paper is silent or garbled are listed in the design notes
of the repository; each is also stated where it is used below.

All functions accept float64 or complex128 numpy arrays (the paper works over
C: A^* is the conjugate transpose, Section 1.1).  The step, X0 and norm helpers
are written with ``@``, ``+`` and ``abs`` only, so they also run on numpy
object arrays of mpmath numbers (the 150-digit reproduction of Table 1).

Parity: every function here is pinned by ``tests/test_oracle.py`` (closed-form
inverses from the generators' factors, the printed Table 1 values, the Penrose
and Drazin equations, exact coefficient identities, Newton-Schulz at p = 2).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

P_ORDER = 18  # order of the method (Eq. hyper18)


# ----------------------------------------------------------------------------
# small helpers (generic over float64 and object arrays)
# ----------------------------------------------------------------------------

def _eye(n: int, like: np.ndarray) -> np.ndarray:
    if like.dtype == object:
        one = like.flat[0] * 0 + 1
        zero = like.flat[0] * 0
        e = np.full((n, n), zero, dtype=object)
        for i in range(n):
            e[i, i] = one
        return e
    return np.eye(n, dtype=like.dtype)


def ct(x: np.ndarray) -> np.ndarray:
    """A^*: the conjugate (Hermitian) transpose (Section 1.1); the transpose
    for real and object arrays."""
    return x.conj().T if np.iscomplexobj(x) else x.T


def fro(x: np.ndarray):
    """Frobenius norm sqrt(sum |x_ij|^2)."""
    if np.iscomplexobj(x):
        return float(np.sqrt((x.real * x.real + x.imag * x.imag).sum()))
    return (x * x).sum() ** 0.5


def norm_inf(x: np.ndarray):
    """Infinity norm: the largest absolute row sum (used in Section 8, Example 1)."""
    return max(abs(v).sum() for v in x)


def trace(x: np.ndarray):
    return sum(x[i, i] for i in range(x.shape[0]))


def matpow(A: np.ndarray, l: int) -> np.ndarray:
    """A^l by l-1 successive products (A^0 = I)."""
    out = _eye(A.shape[0], A)
    for _ in range(l):
        out = out @ A
    return out


# ----------------------------------------------------------------------------
# the coefficients of the factorisation (Section 2)
# ----------------------------------------------------------------------------

def coefficients() -> dict:
    """Closed forms printed in Section 2 for the parameters of Eq. hyper18-33,
    Eq. simplify1 and Eq. simplify2.  Only the factorised reference step and
    the coefficient pins use them; the oracle's own step does not."""
    s93 = math.sqrt(93.0)
    a1 = 5.0 / 496.0 * (31.0 + s93)
    a2 = (3.0 + s93) / 8.0
    a3 = 0.5
    b1 = -5.0 / 496.0 * (s93 - 31.0)
    b2 = (3.0 - s93) / 8.0
    mu = 3.0 / 8.0
    psi = 321.0 / 1984.0
    q = math.sqrt(27.0 - 2.0 * s93)
    c1 = (q + 1.0) / 4.0
    c2 = (1.0 - q) / 4.0
    c3 = (5.0 * s93 - 93.0) / 496.0
    d1 = (-93.0 - 5.0 * s93) / 496.0
    d2 = -s93 / 4.0
    return dict(a1=a1, a2=a2, a3=a3, b1=b1, b2=b2, b3=a3, mu=mu, psi=psi,
                c1=c1, c2=c2, c3=c3, d1=d1, d2=d2)


# ----------------------------------------------------------------------------
# the step
# ----------------------------------------------------------------------------

def choose_side(m: int, n: int) -> str:
    """Which residual to form.  Reading: the paper writes R = I - AX (m x m);
    in exact arithmetic X (I - AX)^j = (I - XA)^j X, so when n < m the same
    iterate comes from the n x n residual I - XA multiplied from the left.
    'right' (the paper's own form) when m <= n, else 'left'."""
    return "right" if m <= n else "left"


def residual(A: np.ndarray, X: np.ndarray, side: str) -> np.ndarray:
    """R = I - A X (right, m x m; Eq. Hyperpower1) or I - X A (left, n x n)."""
    if side == "right":
        P = A @ X
    elif side == "left":
        P = X @ A
    else:
        raise ValueError(side)
    return _eye(P.shape[0], P) - P


def hyperpower_step(A: np.ndarray, X: np.ndarray, p: int = P_ORDER, side: str = "right") -> np.ndarray:
    """One loop of the order-p hyperpower method, formed naively (Eq. Hyperpower1;
    Eq. hyper18 for p = 18): S = I + R + R^2 + ... + R^{p-1} by p-1 successive
    products, then X S (right) or S X (left)."""
    R = residual(A, X, side)
    term = _eye(R.shape[0], R)
    S = term.copy()
    for _ in range(p - 1):
        term = term @ R
        S = S + term
    return X @ S if side == "right" else S @ X


def pm_step(A: np.ndarray, X: np.ndarray, side: str = "right") -> np.ndarray:
    """The factorised seven-product loop of Eq. PM.  Reference for the pin
    'factorised step equals the naive step'; the oracle's solve never calls it."""
    c = coefficients()
    R = residual(A, X, side)
    I = _eye(R.shape[0], R)
    R2 = R @ R
    R4 = R2 @ R2
    M = (I + c["c1"] * R2 + R4) @ (I + c["c2"] * R2 + R4)
    T = M + c["c3"] * R2
    S = M + c["d1"] * R2 + c["d2"] * R4
    Y = (I + R) @ (T @ S + c["mu"] * R2 + c["psi"] * R4)
    return X @ Y if side == "right" else Y @ X


def stabilised_step(A: np.ndarray, X: np.ndarray, p: int = P_ORDER, side: str = "right") -> np.ndarray:
    """Eq. PM-modified: X_{k+1/2} = hyperpower step, X_{k+1} = X_{k+1/2} A X_{k+1/2}."""
    Xh = hyperpower_step(A, X, p, side)
    return Xh @ A @ Xh


# ----------------------------------------------------------------------------
# initial values and scaling (Section 4)
# ----------------------------------------------------------------------------

def x0_moore_penrose(A: np.ndarray, alpha) -> np.ndarray:
    """X0 = alpha A^* (Section 4, Theorem 6.2); alpha A^T for real A."""
    return alpha * ct(A).copy()


def x0_general(G: np.ndarray, alpha) -> np.ndarray:
    """X0 = alpha G (Section 2)."""
    return alpha * G


def drazin_index(A: np.ndarray, max_index: int = 16):
    """ind(A): the smallest nonnegative l with rank(A^{l+1}) = rank(A^l) (the
    definition given with the Drazin initial value in Section 4).  Ranks by
    numpy.linalg.matrix_rank (SVD, its default tolerance).  Returns (l, ranks)
    with ranks[k] = rank(A^k) for k = 0 .. l + 1; l = -1 if it exceeds max_index."""
    n = A.shape[0]
    ranks = [n]
    P = _eye(n, A)
    for k in range(1, max_index + 2):
        P = P @ A
        ranks.append(int(np.linalg.matrix_rank(P)))
        if ranks[k] == ranks[k - 1]:
            return k - 1, ranks
    return -1, ranks


def x0_drazin(A: np.ndarray, l: int, alpha=None) -> np.ndarray:
    """X0 = A^l / Tr(A^{l+1}) (Section 4), or alpha A^l when alpha is given.
    For complex A the trace, and so alpha, is complex as the formula stands."""
    Al = matpow(A, l)
    if alpha is None:
        tr = trace(Al @ A)
        if np.iscomplexobj(A):
            if tr == 0:
                raise ValueError("Tr(A^{l+1}) = 0: no trace scaling")
        elif not tr > 0:
            raise ValueError("Tr(A^{l+1}) must be positive for the trace scaling")
        alpha = 1 / tr
    return alpha * Al


def x0_drazin_normal(A: np.ndarray, l: int, alpha=None) -> np.ndarray:
    """X0 = alpha G with G = A^l (A^{2l+1})^* A^l.  R(G) = R(A^l) and N(G) = N(A^l),
    the range and null space of the Drazin inverse (Section 1.1 names A^D as the
    outer inverse with those subspaces; Theorem 3.1 takes any such G), and GA
    has a real nonnegative spectrum, so the iteration converges whatever the
    eigenvalues of A (X0 = A^l / Tr(A^{l+1}) needs them in a sector).  alpha
    defaults to 1 / sqrt(||GA||_1 ||GA||_inf) <= 1 / ||GA||_2."""
    Al = matpow(A, l)
    G = Al @ ct(matpow(A, 2 * l + 1)) @ Al
    if alpha is None:
        GA = G @ A
        alpha = 1.0 / math.sqrt(float(np.abs(GA).sum(axis=0).max()) * float(np.abs(GA).sum(axis=1).max()))
    return alpha * G


def x0_jacobi(A: np.ndarray, alpha=1.0) -> np.ndarray:
    """X0 = alpha diag(1/a_11, ..., 1/a_nn), the initial matrix of Section 8's
    preconditioning example (Eq. choice3); alpha = 1 as printed."""
    d = np.diag(A)
    if np.any(d == 0):
        raise ValueError("a zero diagonal entry: no Jacobi initial value")
    return alpha * np.diag(1.0 / d)


def alpha_pan_schreiber(sigma_1: float, sigma_r: float) -> float:
    """alpha = 2 / (sigma_1^2 + sigma_r^2) (Section 4), sigma_1 >= sigma_r > 0 the
    extreme nonzero singular values of A (reading of 'eigenvalues of GA' for
    G = A^T: those eigenvalues are sigma_i^2, so the formula squares the
    singular values)."""
    return 2.0 / (sigma_1 ** 2 + sigma_r ** 2)


def alpha_rectangular(A: np.ndarray) -> float:
    """alpha = 1 / (||A||_1 ||A||_inf) (Section 4's recipe for rectangular A)."""
    n1 = float(np.abs(A).sum(axis=0).max())
    ninf = float(np.abs(A).sum(axis=1).max())
    return 1.0 / (n1 * ninf)


def alpha_general(A: np.ndarray, G: np.ndarray) -> float:
    """alpha = 1 / sqrt(||P||_1 ||P||_inf) for X0 = alpha G, P the smaller of GA
    (n x n, when m > n) and AG (m x m): both have the nonzero eigenvalues of GA
    that Section 4's alpha = 2/(lambda_1 + lambda_r) refers to, and the
    spectral radius is at most min(||P||_1, ||P||_inf), so alpha lambda <= 1 for
    every eigenvalue -- inside Theorem 3.1's region when the spectrum of GA is
    real and nonnegative (G = A^*, G = I for A positive definite, weighted
    Moore-Penrose and Bott-Duffin choices).  Reading for general G; Section 4
    gives the Moore-Penrose recipe only."""
    m, n = A.shape
    P = G @ A if m > n else A @ G
    n1 = float(np.abs(P).sum(axis=0).max())
    ninf = float(np.abs(P).sum(axis=1).max())
    return 1.0 / math.sqrt(n1 * ninf)


# ----------------------------------------------------------------------------
# cleanup projections (build-introduced; motivated by Theorems 6.2 and 7.1)
# ----------------------------------------------------------------------------

def cleanup_moore_penrose(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    """X <- (XA)^* X (AX)^*.  With X = A^+ + E in the SVD blocks of Theorem 6.2
    this removes the E12, E21 and E22 blocks to first order (they are the parts
    the iteration does not contract) and leaves A^+ fixed."""
    return ct(X @ A) @ X @ ct(A @ X)


def cleanup_outer(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    """X <- X A X for a general outer inverse A^(2)_{T,S} (the product Section 7
    appends to each loop): it fixes every outer inverse (XAX = X defines them,
    Eq. 1) and removes the first-order error components outside R(X) on the left
    and N(X) on the right.  The Moore-Penrose projection above would move a
    non-Moore-Penrose outer inverse (e.g. a weighted one) away from itself."""
    return X @ A @ X


def cleanup_drazin(A: np.ndarray, X: np.ndarray, l: int) -> np.ndarray:
    """X <- A^l X^{2l+1} A^l; fixes A^D (A^D = A^l (A^D)^{2l+1} A^l) and
    projects an approximate Drazin inverse back onto R(A^l), N(A^l)."""
    Al = matpow(A, l)
    return Al @ matpow(X, 2 * l + 1) @ Al


# ----------------------------------------------------------------------------
# approximate-inverse preconditioners (Section 8, Example 3; the concluding
# remark that one loop of the method already gives a preconditioner)
# ----------------------------------------------------------------------------

def chop(X: np.ndarray, eps: float) -> np.ndarray:
    """Sparsification after each loop in Example 3: every entry of magnitude
    below eps becomes 0; for complex entries the real and imaginary parts are
    tested and zeroed separately (reading of the Chop command used there)."""
    if np.iscomplexobj(X):
        re = np.where(np.abs(X.real) < eps, 0.0, X.real)
        im = np.where(np.abs(X.imag) < eps, 0.0, X.imag)
        return re + 1j * im
    return np.where(np.abs(X) < eps, 0.0, X)


def preconditioner(A: np.ndarray, loops: int = 1, chop_eps: float = 0.0, alpha=1.0):
    """X_k after ``loops`` loops of the order-18 step from the Jacobi X0
    (Eq. choice3), each loop followed by the chop when chop_eps > 0.  Returns
    (X_k, the relative step of every loop, measured before its chop)."""
    X = x0_jacobi(A, alpha)
    side = choose_side(*A.shape)
    steps = []
    for k in range(loops):
        Xn = hyperpower_step(A, X, P_ORDER, side)
        steps.append(stop_measure(Xn, X, k, 1.0, STOP_REL_FRO))
        X = chop(Xn, chop_eps) if chop_eps > 0 else Xn
    return X, steps


# ----------------------------------------------------------------------------
# stopping (Section 4 and the remarks closing Section 6)
# ----------------------------------------------------------------------------

STOP_REL_FRO = 0   # ||X_{k+1} - X_k||_F / ||X_k||_F < tol
STOP_PAPER = 1     # ||X_{k+1} - X_k||_F / (18^k alpha) < tol   (Eq. stopreliable)
STOP_ORDER18 = 2   # relative step < tol (tol = delta, e.g. 1e-2): keep X_{k+1}, no further loop


def stop_measure(Xn: np.ndarray, X: np.ndarray, k: int, alpha: float, mode: int) -> float:
    """Stop measure of loop k (Eq. stopreliable, or the relative step).  A loop
    that leaves X unchanged is at the fixed point of Theorem 3.1's iteration
    and measures 0 under every rule (the relative step would be 0/0 at X = 0,
    the answer when A = 0 or G = 0)."""
    d = float(fro(Xn - X))
    if d == 0.0:
        return 0.0
    if mode in (STOP_REL_FRO, STOP_ORDER18):
        nx = float(fro(X))
        return d / nx if nx > 0 else math.inf
    if mode == STOP_PAPER:
        return d / (P_ORDER ** k * alpha)
    raise ValueError(mode)


@dataclass
class SolveInfo:
    iters: int = 0                    # loops whose result was kept
    loops_run: int = 0                # loops executed (one more when stopped at the minimum)
    stabilised_loops: int = 0
    status: str = "maxiter"           # 'converged' | 'minimum' | 'maxiter' | 'nonfinite'
    history: list = field(default_factory=list)   # stop measure of every loop
    finished: bool = False            # cleanup + one order-2 step applied


def solve(A: np.ndarray, X0: np.ndarray, tol: float = 1e-12, stop: int = STOP_REL_FRO,
          alpha: float = 1.0, max_iter: int = 100, variant: str = "plain",
          switch_tol: float = 1e-3, floor_guard: float = 1e-3, side: str | None = None,
          p: int = P_ORDER, finish: str | None = None, drazin_index: int = 0):
    """Run the iteration from X0 (Theorem 3.1 / Section 7).

    Loop k computes X_{k+1} from X_k with the naive order-p step (plus X A X
    once the stabilised variant is switched on) and the stop measure e_k.
    * e_k < tol: keep X_{k+1}, status 'converged'.  With STOP_ORDER18, tol is a
      threshold delta with delta^18 below the FP64 unit roundoff: by Theorem
      3.1 (F_{k+1} = F_k^18) the loop that produced a step below delta has
      already brought the error to the rounding floor, so no loop is spent
      observing the floor (reading of the order-18 contraction).
    * Plain loops, reading of the first remark closing Section 6: once the
      previous step e_{k-1} was below ``floor_guard`` (the converged regime,
      where order 18 makes e_k of order e_{k-1}^18), a step with
      e_k >= e_{k-1}^2 is not a convergent step but rounding growth (Theorem
      6.2: the null block grows by 18 per loop); keep X_k, status 'minimum'.
    * Stabilised loops (Theorem 7.1: rounding no longer grows): stop when the
      step no longer decreases, e_k >= e_{k-1}; keep X_k, status 'minimum'.
    * Stabilised variant: loops after the first one with e < switch_tol use
      the extra X A X (the Pan-Schreiber switch closing Section 7).
    * ``finish`` ('moore_penrose', 'drazin' or 'outer' for a general G): after
      the loop ends, apply the cleanup projection and one order-2 step of the
      hyperpower family
      (X <- X(I + R), R = I - AX).  The projection removes the blocks Theorem
      6.2 shows are not contracted (E12, E21 persist, E22 grows); its own
      rounding error is first order, which one order-2 step squares.
    max_iter defaults to the paper's 100 (Section 8).
    """
    X, info = _iterate(A, X0, tol, stop, alpha, max_iter, variant, switch_tol, floor_guard,
                       side or choose_side(*A.shape), p)
    if finish is not None and info.status != "nonfinite":
        if finish == "moore_penrose":
            Xc = cleanup_moore_penrose(A, X)
        elif finish == "drazin":
            Xc = cleanup_drazin(A, X, drazin_index)
        elif finish == "outer":
            Xc = cleanup_outer(A, X)
        else:
            raise ValueError(finish)
        X = hyperpower_step(A, Xc, 2, side or choose_side(*A.shape))
        info.finished = True
    return X, info


def _iterate(A, X0, tol, stop, alpha, max_iter, variant, switch_tol, floor_guard, side, p):
    info = SolveInfo()
    X = X0
    prev = math.inf
    stabilise = False
    for k in range(max_iter):
        stabilised_now = stabilise
        if stabilised_now:
            Xn = stabilised_step(A, X, p, side)
            info.stabilised_loops += 1
        else:
            Xn = hyperpower_step(A, X, p, side)
        e = stop_measure(Xn, X, k, alpha, stop)
        info.loops_run = k + 1
        info.history.append(e)
        if not math.isfinite(e):
            info.status = "nonfinite"
            info.iters = k
            return X, info
        if e < tol:
            info.status = "converged"
            info.iters = k + 1
            return Xn, info
        stalled = (e >= prev) if stabilised_now else (prev < floor_guard and e >= prev * prev)
        if stalled:
            info.status = "minimum"
            info.iters = k
            return X, info
        if variant == "stabilised" and e < switch_tol:
            stabilise = True
        prev = e
        X = Xn
    info.iters = max_iter
    return X, info


# ----------------------------------------------------------------------------
# residual checks (Eq. 1; the Penrose and Drazin equations; Eq. COC)
# ----------------------------------------------------------------------------

def penrose_residuals(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Relative Frobenius residuals of the four Penrose equations:
    ||AXA - A||/||A||, ||XAX - X||/||X||, ||(AX)^* - AX||/||AX||, ||(XA)^* - XA||/||XA||."""
    AX = A @ X
    XA = X @ A
    return np.array([
        float(fro(AX @ A - A) / fro(A)),
        float(fro(X @ AX - X) / fro(X)),
        float(fro(ct(AX) - AX) / fro(AX)),
        float(fro(ct(XA) - XA) / fro(XA)),
    ])


def drazin_residuals(A: np.ndarray, X: np.ndarray, l: int) -> np.ndarray:
    """Relative residuals of XAX = X, AX = XA and A^{l+1} X = A^l."""
    Al = matpow(A, l)
    AX = A @ X
    return np.array([
        float(fro(X @ AX - X) / fro(X)),
        float(fro(AX - X @ A) / fro(AX)),
        float(fro(Al @ AX - Al) / fro(Al)),
    ])


def coc(d: list) -> list:
    """Computational order of convergence (Eq. COC, Section 8).  The printed
    fraction is garbled; read as rho_k = ln(d_{k+1}/d_k) / ln(d_k/d_{k-1}) with
    d_k = ||X_k - X_{k-1}||_inf."""
    out = []
    for k in range(1, len(d) - 1):
        out.append(math.log(d[k + 1] / d[k]) / math.log(d[k] / d[k - 1]))
    return out


def relative_error(X: np.ndarray, Xref: np.ndarray) -> float:
    return float(fro(X - Xref) / fro(Xref))
