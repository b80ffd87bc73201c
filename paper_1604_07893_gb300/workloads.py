"""Seeded synthetic inputs shaped like the paper's test families.

This module only draws matrices; it contains none of the iteration's
arithmetic.  Both the CUDA path (through the tests and the benchmark) and the
FP64 oracle consume what it returns, so it is the one piece of code the two
sides share.

Families (Section 8 of the paper uses a Drazin example, rectangular
ill-conditioned Moore-Penrose problems and preconditioning of a large matrix):

* ``rectangular``  A = U diag(s) V^T with Haar-distributed orthonormal U, V,
  optionally rank-deficient (Moore-Penrose problems, Section 8 Example 2).
* ``drazin_index2`` A = P blockdiag(C, N) P^{-1} with C nonsingular in real
  Schur form and N made of 2x2 nilpotent Jordan blocks (index 2; Section 4
  X0 recipe for the Drazin inverse).
* ``spd``          A = Q diag(lambda) Q^T (the nonsingular / preconditioner
  family, Section 8 Example 3 stand-in).
* ``uneven_batch`` many independent rectangular problems of random shape.
* ``poisson_arrivals`` request arrival times for the serving workload.
* ``hilbert``      H_ij = 1/(i+j-1) (Section 8 Example 2).
* ``subspace_projector`` and ``spd``/``hpd_complex`` weights: the G of the
  weighted Moore-Penrose (G = N^{-1} A^* M) and Bott-Duffin (G = P_L)
  inverses, outer inverses Section 1.1 lists among the A^(2)_{T,S}.
* ``grid_operator``: a shifted five-point operator on a k x k grid, real or
  complex (the sparse-system stand-in for the preconditioning example of
  Section 8, whose MatrixMarket matrix is not used).
* ``rectangular_complex``, ``drazin_complex``, ``hpd_complex``: the same
  families over C (the paper states the method for complex matrices, with
  A^* the conjugate transpose; Section 1.1), complex128 arrays.

Every function takes an integer seed and returns float64 numpy arrays plus the
factors from which the exact answer has a closed form (the tests use those
factors to pin the oracle).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def haar_orthogonal(rng: np.random.Generator, n: int, k: int | None = None) -> np.ndarray:
    """First ``k`` columns of a Haar-distributed n x n orthogonal matrix.

    QR of a standard Gaussian matrix with the signs of R's diagonal folded into
    Q (Mezzadri's correction), which makes the distribution exactly Haar.
    """
    k = n if k is None else k
    g = rng.standard_normal((n, k))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


@dataclass
class Rectangular:
    A: np.ndarray      # m x n
    U: np.ndarray      # m x r, orthonormal columns
    s: np.ndarray      # r singular values, descending
    V: np.ndarray      # n x r, orthonormal columns


def rectangular(m: int, n: int, rank: int | None = None, s_max: float = 1.0,
                s_min: float = 1e-2, seed: int = 0, spacing: str = "log") -> Rectangular:
    """A = U diag(s) V^T with Haar U (m x r), V (n x r).

    ``spacing='log'``: s log-spaced from s_max down to s_min.
    ``spacing='loguniform'``: s = sorted 10**Uniform(log10 s_min, log10 s_max).
    """
    r = min(m, n) if rank is None else rank
    if not (0 < r <= min(m, n)):
        raise ValueError("rank must be in [1, min(m, n)]")
    rng = np.random.default_rng(seed)
    U = haar_orthogonal(rng, m, r)
    V = haar_orthogonal(rng, n, r)
    if spacing == "log":
        s = np.logspace(math.log10(s_max), math.log10(s_min), r)
    elif spacing == "loguniform":
        s = np.sort(10.0 ** rng.uniform(math.log10(s_min), math.log10(s_max), r))[::-1].copy()
    else:
        raise ValueError(spacing)
    A = (U * s) @ V.T
    return Rectangular(A=np.ascontiguousarray(A), U=U, s=s, V=V)


@dataclass
class Drazin:
    A: np.ndarray      # n x n, index 2
    P: np.ndarray      # similarity
    C: np.ndarray      # nonsingular block (real Schur form)
    N: np.ndarray      # nilpotent block, N^2 = 0
    eig: np.ndarray    # eigenvalues of C (complex)


def drazin_index2(n: int, n_nil: int, seed: int = 2, r_min: float = 0.5, r_max: float = 2.0,
                  sector: float = math.pi / 8, p_scale: float | None = None,
                  upper: float = 0.1) -> Drazin:
    """A = P blockdiag(C, N) P^{-1}, ind(A) = 2 when n_nil > 0.

    C (n - n_nil square) is quasi-upper-triangular: 2x2 rotation-scaling blocks
    [[a, b], [-b, a]] for conjugate pairs r e^{+-i theta} (one real 1x1 block if
    the size is odd), with r uniform-in-area on [r_min, r_max] and
    |theta| <= sector, plus a small strictly upper part of scale ``upper/sqrt(n)``.
    N consists of 2x2 Jordan blocks [[0, 1], [0, 0]] (n_nil must be even).
    P = I + p_scale * Gaussian, with p_scale = 0.1/sqrt(n) by default.
    """
    if n_nil % 2 or n_nil > n:
        raise ValueError("n_nil must be even and <= n")
    rng = np.random.default_rng(seed)
    nc = n - n_nil
    C = np.zeros((nc, nc))
    eig = []
    i = 0
    while i < nc:
        r = math.sqrt(rng.uniform(r_min ** 2, r_max ** 2))
        if nc - i >= 2:
            th = rng.uniform(-sector, sector)
            a, b = r * math.cos(th), r * math.sin(th)
            C[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
            eig += [complex(a, b), complex(a, -b)]
            i += 2
        else:
            C[i, i] = r
            eig.append(complex(r, 0.0))
            i += 1
    if nc > 0:
        T = np.triu(rng.standard_normal((nc, nc)) * (upper / math.sqrt(max(n, 1))), 2)
        # keep the 2x2 diagonal blocks intact: only entries strictly above them
        C = C + T
    N = np.zeros((n_nil, n_nil))
    for j in range(0, n_nil, 2):
        N[j, j + 1] = 1.0
    if p_scale is None:
        p_scale = 0.1 / math.sqrt(n)
    P = np.eye(n) + p_scale * rng.standard_normal((n, n))
    B = np.zeros((n, n))
    B[:nc, :nc] = C
    B[nc:, nc:] = N
    A = P @ B @ np.linalg.inv(P)
    return Drazin(A=np.ascontiguousarray(A), P=P, C=C, N=N, eig=np.array(eig))


@dataclass
class SPD:
    A: np.ndarray
    Q: np.ndarray
    lam: np.ndarray


def spd(n: int, lam_min: float = 1e-3, lam_max: float = 1.0, seed: int = 5) -> SPD:
    """A = Q diag(lambda) Q^T, Q Haar, lambda log-spaced in [lam_min, lam_max]."""
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(rng, n)
    lam = np.logspace(math.log10(lam_max), math.log10(lam_min), n)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    return SPD(A=np.ascontiguousarray(A), Q=Q, lam=lam)


def uneven_shapes(count: int, seed: int = 3, m_lo: int = 32, m_hi: int = 512,
                  n_lo: int = 16) -> list[tuple[int, int]]:
    """(m, n) pairs with m ~ U{m_lo..m_hi}, n ~ U{n_lo..m}."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    return [(int(m), int(rng.integers(n_lo, m + 1))) for m in ms]


def uneven_batch(count: int, seed: int = 3, s_min: float = 1e-3, m_lo: int = 32,
                 m_hi: int = 512, n_lo: int = 16) -> list[Rectangular]:
    """Independent full-rank problems, singular values log-uniform in [s_min, 1]."""
    shapes = uneven_shapes(count, seed, m_lo, m_hi, n_lo)
    return [rectangular(m, n, None, 1.0, s_min, seed=seed * 1_000_003 + i, spacing="loguniform")
            for i, (m, n) in enumerate(shapes)]


def poisson_arrivals(rate_per_s: float, count: int, seed: int = 5) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: cumulative exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def serving_sizes(count: int, seed: int = 5,
                  sizes=(256, 512, 1024, 2048, 4096, 8192),
                  weights=(0.40, 0.25, 0.15, 0.10, 0.07, 0.03)) -> np.ndarray:
    rng = np.random.default_rng(seed + 1)
    w = np.asarray(weights, dtype=float)
    return rng.choice(np.asarray(sizes), size=count, p=w / w.sum())


def hilbert(m: int, n: int) -> np.ndarray:
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, n + 1)[None, :]
    return 1.0 / (i + j - 1.0)



def householder_orthogonal(rng: np.random.Generator, n: int, k: int | None = None,
                           reflectors: int = 3) -> np.ndarray:
    """First k columns of H_1 H_2 ... H_r, H_i = I - 2 v_i v_i^T / (v_i^T v_i) with
    Gaussian v_i: a dense seeded orthogonal matrix formed in O(r n^2) (used where
    a workload needs many or very large orthogonal factors and does not ask for
    Haar ones)."""
    k = n if k is None else k
    Q = np.eye(n)[:, :k].copy()
    for _ in range(reflectors):
        v = rng.standard_normal(n)
        v /= np.linalg.norm(v)
        Q -= 2.0 * np.outer(v, v @ Q)
    return Q


def uneven_batch_fast(count: int, seed: int = 3, s_min: float = 1e-3, m_lo: int = 32,
                      m_hi: int = 512, n_lo: int = 16) -> list[Rectangular]:
    """The uneven batch family with Householder-product factors: A = U diag(s) V^T,
    m ~ U{m_lo..m_hi}, n ~ U{n_lo..m}, rank n, s log-uniform in [s_min, 1]."""
    shapes = uneven_shapes(count, seed, m_lo, m_hi, n_lo)
    out = []
    for i, (m, n) in enumerate(shapes):
        rng = np.random.default_rng(seed * 1_000_003 + i)
        U = householder_orthogonal(rng, m, n)
        V = householder_orthogonal(rng, n, n)
        s = np.sort(10.0 ** rng.uniform(math.log10(s_min), 0.0, n))[::-1].copy()
        out.append(Rectangular(A=np.ascontiguousarray((U * s) @ V.T), U=U, s=s, V=V))
    return out


def spd_fast(n: int, lam_min: float = 1e-3, lam_max: float = 1.0, seed: int = 5):
    """Factors of the SPD family with a Householder-product Q (A itself is formed
    by the caller, e.g. on the device): returns (Q, lambda)."""
    rng = np.random.default_rng(seed)
    Q = householder_orthogonal(rng, n)
    lam = np.logspace(math.log10(lam_max), math.log10(lam_min), n)
    return Q, lam


# ---------------------------------------------------------------- complex families

def haar_unitary(rng: np.random.Generator, n: int, k: int | None = None) -> np.ndarray:
    """First ``k`` columns of a Haar-distributed n x n unitary matrix: QR of a
    complex Gaussian matrix (independent N(0, 1/2) real and imaginary parts)
    with the phases of R's diagonal folded into Q (Mezzadri's correction)."""
    k = n if k is None else k
    g = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))) / math.sqrt(2.0)
    q, r = np.linalg.qr(g)
    d = np.diag(r)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return q * ph


def rectangular_complex(m: int, n: int, rank: int | None = None, s_max: float = 1.0,
                        s_min: float = 1e-2, seed: int = 0) -> Rectangular:
    """A = U diag(s) V^* with Haar unitary columns U (m x r), V (n x r) and s
    log-spaced from s_max down to s_min."""
    r = min(m, n) if rank is None else rank
    if not (0 < r <= min(m, n)):
        raise ValueError("rank must be in [1, min(m, n)]")
    rng = np.random.default_rng(seed)
    U = haar_unitary(rng, m, r)
    V = haar_unitary(rng, n, r)
    s = np.logspace(math.log10(s_max), math.log10(s_min), r)
    A = (U * s) @ V.conj().T
    return Rectangular(A=np.ascontiguousarray(A), U=U, s=s, V=V)


def drazin_complex(n: int, n_nil: int, seed: int = 2, r_min: float = 0.5, r_max: float = 2.0,
                   sector: float = math.pi / 8, p_scale: float | None = None,
                   upper: float = 0.1) -> Drazin:
    """A = P blockdiag(C, N) P^{-1} over C, ind(A) = 2 when n_nil > 0.

    C (n - n_nil square) is upper triangular with eigenvalues r e^{i theta},
    r uniform in area on [r_min, r_max], |theta| <= sector drawn independently
    (the spectrum is not closed under conjugation), plus a strictly upper part of
    complex Gaussian entries of scale ``upper/sqrt(n)``.  N: 2x2 Jordan blocks.
    P = I + p_scale * complex Gaussian, p_scale = 0.1/sqrt(n) by default."""
    if n_nil % 2 or n_nil > n:
        raise ValueError("n_nil must be even and <= n")
    rng = np.random.default_rng(seed)
    nc = n - n_nil
    r = np.sqrt(rng.uniform(r_min ** 2, r_max ** 2, nc))
    th = rng.uniform(-sector, sector, nc)
    eig = r * np.exp(1j * th)
    g = (rng.standard_normal((nc, nc)) + 1j * rng.standard_normal((nc, nc))) / math.sqrt(2.0)
    C = np.diag(eig) + np.triu(g, 1) * (upper / math.sqrt(max(n, 1)))
    N = np.zeros((n_nil, n_nil), dtype=complex)
    for j in range(0, n_nil, 2):
        N[j, j + 1] = 1.0
    if p_scale is None:
        p_scale = 0.1 / math.sqrt(n)
    gp = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    P = np.eye(n) + p_scale * gp
    B = np.zeros((n, n), dtype=complex)
    B[:nc, :nc] = C
    B[nc:, nc:] = N
    A = P @ B @ np.linalg.inv(P)
    return Drazin(A=np.ascontiguousarray(A), P=P, C=C, N=N, eig=eig)


def hpd_complex(n: int, lam_min: float = 1e-3, lam_max: float = 1.0, seed: int = 5) -> SPD:
    """A = Q diag(lambda) Q^*, Q Haar unitary, lambda log-spaced in [lam_min, lam_max]."""
    rng = np.random.default_rng(seed)
    Q = haar_unitary(rng, n)
    lam = np.logspace(math.log10(lam_max), math.log10(lam_min), n)
    A = (Q * lam) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    return SPD(A=np.ascontiguousarray(A), Q=Q, lam=lam)


def grid_operator(k: int, shift: complex = 0.5 + 0.5j, jitter: float = 0.05, seed: int = 7,
                  complex_: bool = True) -> np.ndarray:
    """Dense n x n (n = k^2) matrix of a five-point operator on a k x k grid:
    diagonal 4 + shift, -1 to each grid neighbour, every coupling and diagonal
    entry perturbed by a factor (1 + jitter * g) with g standard Gaussian
    (complex Gaussian when ``complex_``; the real part of ``shift`` otherwise).
    Sparse (at most five nonzeros a row) but not banded."""
    rng = np.random.default_rng(seed)
    n = k * k

    def g(size):
        if complex_:
            return (rng.standard_normal(size) + 1j * rng.standard_normal(size)) / math.sqrt(2.0)
        return rng.standard_normal(size)

    A = np.zeros((n, n), dtype=np.complex128 if complex_ else np.float64)
    s = shift if complex_ else float(np.real(shift))
    idx = np.arange(n)
    A[idx, idx] = (4.0 + s) * (1.0 + jitter * g(n))
    for di, dj in ((0, 1), (1, 0), (0, -1), (-1, 0)):
        for i in range(k):
            for j in range(k):
                ii, jj = i + di, j + dj
                if 0 <= ii < k and 0 <= jj < k:
                    A[i * k + j, ii * k + jj] = -1.0 * (1.0 + jitter * g(1)[0])
    return A


def subspace_projector(n: int, k: int, seed: int = 13, complex_: bool = False):
    """Orthogonal projector P_L = Q Q^* onto a Haar-random k-dimensional subspace
    L of R^n (C^n when complex_); returns (P_L, Q)."""
    rng = np.random.default_rng(seed)
    Q = haar_unitary(rng, n, k) if complex_ else haar_orthogonal(rng, n, k)
    P = Q @ Q.conj().T
    return np.ascontiguousarray(P), Q
