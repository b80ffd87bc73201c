"""CPU model of the product classes of the GPU path, for choosing and checking
precision schedules of the order-18 iteration.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests call it.  It shares no code with the CUDA path (numpy only) and
models the *arithmetic* of each product class from its definition, so that a
schedule (which loops run in which class) can be tried on the CPU before it is
trusted on the GPU:

* ``round_bits(x, p)``: x rounded to nearest (ties to even) with p significant
  bits -- BF16 is p = 8 (an 8-bit exponent and 7 stored fraction bits), FP32
  p = 24.  Exponent range is not modelled (every value here is far inside it).
* ``e4m3(x)``: the FP8 E4M3 format (4 exponent bits, bias 7, 3 fraction bits,
  largest finite 448, subnormal spacing 2^-9), round to nearest even,
  saturating at +-448.
* ``slice_product(A, B, S, L)``: the exact-slice product.  Each row of A (each
  column of B) is scaled by the power of two 2^-e that brings its largest entry
  into [1/2, 1), rounded to a T = 8S - 1 bit fixed-point integer U (ties
  away from zero), and U is cut into S balanced base-256 digits q_s in
  [-128, 128] (from the least significant byte up, a byte >= 128 becomes
  byte - 256 and carries 1).  Slice s holds q_s 2^(8(S-1-s) - T) 2^e.  The
  product keeps the slice pairs with s + t <= L; each pair's product is exact
  here (integers below 2^53 in a common unit).  S = 7, L = 6 is the
  FP64-class product (55 bits, 28 pairs); S = 4, L = 3 the FP32-class product
  (31 bits, 10 pairs).
* ``bf16_product``: both operands rounded to BF16, products accumulated in
  FP32 (modelled as the exact product of the rounded operands, rounded once
  to FP32).
* ``fp8_product``: per-tensor scaled E4M3 operands (scale = 448 / amax), FP32
  accumulation, scales divided out.

The loop, the stabilising product, the projection and the order-2 step below
are written in the grouping the GPU path evaluates (each product is one call
of the class's ``mul``; linear combinations and the update X + D X in FP64):
R = I - XA (or I - AX), R2 = RR, R4 = R2R2, L1 = I + c1R2 + R4,
L2 = I + c2R2 + R4, M = L1L2, T = M + c3R2, S = M + d1R2 + d2R4,
Z = TS + mu R2 + psi R4, D = RZ + Z - I, X' = X + DX (Eq. PM, Section 2), so
X' = X (I + R)(TS + mu R2 + psi R4) in exact arithmetic.

Pinned by ``tests/test_precision_model.py`` (rounding against torch's BF16
conversion and hand cases, the slice digits against their definition, the
slice product against exact rational products within its truncation bound).
"""

from __future__ import annotations

import math

import numpy as np

from . import hyperpower as H


# ----------------------------------------------------------------------------
# number formats
# ----------------------------------------------------------------------------

def round_bits(x: np.ndarray, p: int) -> np.ndarray:
    """x rounded to nearest with p significant bits, ties to even."""
    x = np.asarray(x, dtype=np.float64)
    f, e = np.frexp(x)                       # x = f 2^e, 1/2 <= |f| < 1
    return np.ldexp(np.rint(np.ldexp(f, p)), e - p)   # rint: ties to even


def bf16(x: np.ndarray) -> np.ndarray:
    """BF16 round to nearest even (8 significant bits)."""
    return round_bits(x, 8)


def fp32(x: np.ndarray) -> np.ndarray:
    """FP32 round to nearest even (24 significant bits)."""
    return round_bits(x, 24)


E4M3_MAX = 448.0


def e4m3(x: np.ndarray) -> np.ndarray:
    """FP8 E4M3: 4 significant bits for normal values (|x| >= 2^-6), a fixed
    spacing of 2^-9 below that, round to nearest even, saturating at 448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    normal = round_bits(x, 4)
    sub = np.ldexp(np.rint(np.ldexp(x, 9)), -9)
    y = np.where(a >= 2.0 ** -6, normal, sub)
    return np.clip(y, -E4M3_MAX, E4M3_MAX)


# ----------------------------------------------------------------------------
# the exact-slice product
# ----------------------------------------------------------------------------

def _grid_exponents(X: np.ndarray, axis: int) -> np.ndarray:
    """e per row (axis=1) or column (axis=0) with max |x| in [2^(e-1), 2^e); 0
    for an all-zero line."""
    mx = np.max(np.abs(X), axis=axis, keepdims=True)
    _, e = np.frexp(mx)
    return np.where(mx > 0, e, 0)


def digits(X: np.ndarray, S: int, axis: int):
    """The balanced base-256 digits of X scaled per line: returns (q, e) with
    q[s] integer arrays (most significant first, |q| <= 128) and e the line
    exponents, such that X ~= sum_s q[s] 2^(8(S-1-s) - T) 2^e, T = 8S - 1."""
    T = 8 * S - 1
    e = _grid_exponents(X, axis)
    U = np.floor(np.abs(X) * np.exp2(T - e) + 0.5).astype(np.int64)   # <= 2^T
    sign = np.where(X < 0, -1, 1)
    q = [None] * S
    carry = np.zeros_like(U)
    for b in range(S):                       # from the least significant byte
        d = ((U >> (8 * b)) & 0xFF) + carry
        if b < S - 1:
            up = d >= 128
            d = np.where(up, d - 256, d)
            carry = up.astype(np.int64)
        q[S - 1 - b] = sign * d
    return q, e


def slices(X: np.ndarray, S: int, axis: int) -> list:
    """The S slices of X (row-normalised for axis=1, column-normalised for axis=0)."""
    q, e = digits(X, S, axis)
    T = 8 * S - 1
    return [q[s] * np.exp2(8 * (S - 1 - s) - T) * np.exp2(e) for s in range(S)]


def slice_product(A: np.ndarray, B: np.ndarray, S: int, L: int) -> np.ndarray:
    """sum over slice pairs s + t <= L of A_s B_t (rows of A, columns of B)."""
    As = slices(A, S, 1)
    Bs = slices(B, S, 0)
    C = np.zeros((A.shape[0], B.shape[1]))
    for s in range(S):
        for t in range(S):
            if s + t <= L:
                C += As[s] @ Bs[t]
    return C


def bf16_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    return fp32(bf16(A) @ bf16(B))


def fp8_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Per-tensor scaled E4M3 operands, FP32 accumulation."""
    sa = E4M3_MAX / max(float(np.max(np.abs(A))), 1e-300)
    sb = E4M3_MAX / max(float(np.max(np.abs(B))), 1e-300)
    return fp32(e4m3(A * sa) @ e4m3(B * sb)) / (sa * sb)


CLASSES = {
    "fp64": lambda A, B: A @ B,
    "fp64_class": lambda A, B: slice_product(A, B, 7, 6),
    "fp32_class": lambda A, B: slice_product(A, B, 4, 3),
    "bf16": bf16_product,
    "fp8": fp8_product,
}


# ----------------------------------------------------------------------------
# the loop and the finish in the GPU path's grouping
# ----------------------------------------------------------------------------

def pm_loop(A: np.ndarray, X: np.ndarray, mul, side: str) -> np.ndarray:
    """One loop of Eq. PM with every product formed by ``mul``."""
    c = H.coefficients()
    if side == "left":
        R = np.eye(X.shape[0]) - mul(X, A)
    else:
        R = np.eye(A.shape[0]) - mul(A, X)
    I = np.eye(R.shape[0])
    R2 = mul(R, R)
    R4 = mul(R2, R2)
    L1 = R4 + c["c1"] * R2 + I
    L2 = R4 + c["c2"] * R2 + I
    M = mul(L1, L2)
    T = M + c["c3"] * R2
    S = M + c["d1"] * R2 + c["d2"] * R4
    Z = mul(T, S) + c["mu"] * R2 + c["psi"] * R4
    D = mul(R, Z) + Z - I
    return X + (mul(D, X) if side == "left" else mul(X, D))


def xax(A: np.ndarray, X: np.ndarray, mul, side: str) -> np.ndarray:
    """X A X with the smaller square in the middle (Eq. PM-modified's product)."""
    if side == "left":
        return mul(mul(X, A), X)
    return mul(X, mul(A, X))


def order2_step(A: np.ndarray, X: np.ndarray, mul, side: str) -> np.ndarray:
    """One step of the hyperpower family with p = 2 (Eq. hyper): X + (I - XA) X
    (left residual) or X + X (I - AX) (right), both products formed by ``mul``."""
    if side == "left":
        return X + mul(np.eye(X.shape[0]) - mul(X, A), X)
    return X + mul(X, np.eye(A.shape[0]) - mul(A, X))


def finish_moore_penrose(A: np.ndarray, X: np.ndarray, mul, side: str, step: str = "order2") -> np.ndarray:
    """The build's finish: X <- (XA)^T X (AX)^T, then one order-2 step
    X + (I - XA) X (or X + X (I - AX)), or one order-18 loop (step='order18')."""
    P = mul(X, A)
    Q = mul(A, X)
    X = mul(mul(P.T, X), Q.T)
    if step == "order18":
        return pm_loop(A, X, mul, side)
    if side == "left":
        return X + mul(np.eye(X.shape[0]) - mul(X, A), X)
    return X + mul(X, np.eye(A.shape[0]) - mul(A, X))


def finish_drazin(A: np.ndarray, X: np.ndarray, l: int, mul, step: str = "order2") -> np.ndarray:
    """The Drazin finish: X <- A^l X^{2l+1} A^l, then one order-2 step
    X + X (I - AX) (or one order-18 loop)."""
    Al = A
    for _ in range(l - 1):
        Al = mul(Al, A)
    V = X
    for _ in range(2 * l):
        V = mul(V, X)
    X = mul(mul(Al, V), Al)
    if step == "order18":
        return pm_loop(A, X, mul, "right")
    return X + mul(X, np.eye(A.shape[0]) - mul(A, X))


def run_schedule(A: np.ndarray, X0: np.ndarray, classes: list, finish: str | None = "order2",
                 finish_class: str = "fp64_class", stabilise_from: int | None = None,
                 drazin_index: int = 0):
    """Loops k = 0 .. len(classes)-1 with the products of class classes[k]
    (plus X A X in loops >= stabilise_from), then the finish in finish_class
    (the Drazin finish when drazin_index > 0, else the Moore-Penrose one).
    Returns (X, relative steps of the loops)."""
    side = "right" if drazin_index else H.choose_side(*A.shape)
    X = X0
    steps = []
    for k, cls in enumerate(classes):
        mul = CLASSES[cls]
        Xn = pm_loop(A, X, mul, side)
        if stabilise_from is not None and k >= stabilise_from:
            Xn = xax(A, Xn, mul, side)
        nx = np.linalg.norm(X)
        steps.append(float(np.linalg.norm(Xn - X) / nx) if nx > 0 else math.inf)
        X = Xn
        if not np.all(np.isfinite(X)):
            return X, steps
    if finish is not None:
        if drazin_index:
            X = finish_drazin(A, X, drazin_index, CLASSES[finish_class], finish)
        else:
            X = finish_moore_penrose(A, X, CLASSES[finish_class], side, finish)
    return X, steps
