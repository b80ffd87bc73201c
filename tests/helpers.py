"""Small helpers shared by the tests (fixture loading, closed-form answers)."""
import os
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def example1(kind="float"):
    """The printed 12 x 12 matrix of Section 8, Example 1 (tests/golden)."""
    path = os.path.join(ROOT, "tests", "golden", "example1_drazin.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    if kind == "float":
        return np.array([[float(Fraction(x)) for x in r] for r in rows])
    if kind == "fraction":
        return [[Fraction(x) for x in r] for r in rows]
    raise ValueError(kind)


def pinv_closed_form(w):
    """A^+ = V diag(1/s) U^* from the generator's factors."""
    return (w.V / w.s) @ w.U.conj().T


def drazin_closed_form(d):
    """A^D = P blockdiag(C^{-1}, 0) P^{-1} from the generator's factors."""
    n = d.A.shape[0]
    nc = d.C.shape[0]
    B = np.zeros((n, n), dtype=d.A.dtype)
    if nc:
        B[:nc, :nc] = np.linalg.inv(d.C)
    return d.P @ B @ np.linalg.inv(d.P)


def spd_inverse(s):
    return (s.Q / s.lam) @ s.Q.conj().T


def rel(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))
