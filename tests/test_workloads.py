"""CPU checks of the seeded input generators against the recipes they state
(shapes, ranks, spectra, structure): the inputs both the oracle and the GPU
path consume."""

import math

import numpy as np
import pytest

from paper_1604_07893_gb300 import workloads as W


def test_rectangular_complex_recipe():
    w = W.rectangular_complex(40, 30, 20, 1.0, 1e-3, seed=4)
    assert w.A.shape == (40, 30) and w.A.dtype == np.complex128
    assert np.allclose(w.U.conj().T @ w.U, np.eye(20), atol=1e-13)
    assert np.allclose(w.V.conj().T @ w.V, np.eye(20), atol=1e-13)
    s = np.linalg.svd(w.A, compute_uv=False)
    assert np.allclose(s[:20], np.logspace(0, -3, 20), rtol=1e-10)
    assert s[20] < 1e-13
    assert np.abs(w.A.imag).max() > 0.1          # genuinely complex
    assert np.array_equal(w.A, W.rectangular_complex(40, 30, 20, 1.0, 1e-3, seed=4).A)   # seeded


def test_drazin_complex_recipe():
    d = W.drazin_complex(50, 10, seed=5)
    assert np.linalg.matrix_rank(d.A) == 45 and np.linalg.matrix_rank(d.A @ d.A) == 40
    assert np.all(np.abs(np.angle(d.eig)) <= math.pi / 8 + 1e-12)
    r = np.abs(d.eig)
    assert r.min() >= 0.5 - 1e-12 and r.max() <= 2.0 + 1e-12
    assert not np.allclose(np.sort_complex(d.eig), np.sort_complex(d.eig.conj()))   # no conjugate pairs
    lam = np.linalg.eigvals(d.A)
    nz = lam[np.abs(lam) > 1e-6]
    assert np.allclose(np.sort_complex(nz), np.sort_complex(d.eig), atol=1e-8)


def test_grid_operator_recipe():
    k = 9
    A = W.grid_operator(k, seed=7)
    n = k * k
    assert A.shape == (n, n) and A.dtype == np.complex128
    assert (np.count_nonzero(A, axis=1) <= 5).all()
    # couplings only between grid neighbours
    rows, cols = np.nonzero(A)
    for i, j in zip(rows, cols):
        di, dj = divmod(i, k), divmod(j, k)
        assert abs(di[0] - dj[0]) + abs(di[1] - dj[1]) <= 1
    # the Jacobi iteration matrix contracts (the preconditioner family needs it)
    L0 = np.eye(n) - np.diag(1.0 / np.diag(A)) @ A
    assert max(abs(np.linalg.eigvals(L0))) < 1.0
    Ar = W.grid_operator(k, seed=7, complex_=False)
    assert Ar.dtype == np.float64 and (np.count_nonzero(Ar, axis=1) <= 5).all()


def test_hpd_complex_and_projector_recipes():
    s = W.hpd_complex(20, 1e-2, 1.0, seed=6)
    assert np.allclose(s.A, s.A.conj().T, atol=1e-15)
    assert np.allclose(np.sort(np.linalg.eigvalsh(s.A)), np.sort(s.lam), rtol=1e-10)
    P, Q = W.subspace_projector(20, 7, seed=8)
    assert np.allclose(P @ P, P, atol=1e-14) and np.allclose(P, P.T, atol=1e-15)
    assert round(np.trace(P)) == 7


@pytest.mark.parametrize("m,n", [(64, 48), (48, 64)])
def test_rectangular_recipe(m, n):
    w = W.rectangular(m, n, None, 1.0, 1e-2, seed=0)
    assert np.allclose(np.linalg.svd(w.A, compute_uv=False), np.logspace(0, -2, min(m, n)), rtol=1e-10)
