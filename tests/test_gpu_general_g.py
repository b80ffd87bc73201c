"""GPU parity of outer inverses through a caller G (Section 1.1 lists them
among the A^(2)_{T,S}): the weighted Moore-Penrose inverse (G = N^{-1} A^* M)
and the Bott-Duffin inverse (G = P_L), with the general-G alpha recipe
(alpha = 0) and the X A X finish, on the single-solve and batched paths.

References: the oracle (same alpha recipe, same finish) and the closed forms
N^{-1/2} (M^{1/2} A N^{-1/2})^+ M^{1/2} and P_L (A P_L + P_{L^perp})^{-1};
FP64-finished bar 1e-9."""

import ctypes as C

import numpy as np
import pytest

from oracle import hyperpower as H
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import rel

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


def _pow(s, p):
    return (s.Q * s.lam ** p) @ s.Q.conj().T


def weighted_problem(m, n, r, seed, complex_=False):
    if complex_:
        w = W.rectangular_complex(m, n, r, 1.0, 1e-3, seed=seed)
        Ms, Ns = W.hpd_complex(m, 0.2, 5.0, seed=seed + 1), W.hpd_complex(n, 0.5, 2.0, seed=seed + 2)
    else:
        w = W.rectangular(m, n, r, 1.0, 1e-3, seed=seed)
        Ms, Ns = W.spd(m, 0.2, 5.0, seed=seed + 1), W.spd(n, 0.5, 2.0, seed=seed + 2)
    A = w.A
    G = np.ascontiguousarray(_pow(Ns, -1.0) @ H.ct(A) @ Ms.A)
    ref = _pow(Ns, -0.5) @ np.linalg.pinv(_pow(Ms, 0.5) @ A @ _pow(Ns, -0.5), rcond=1e-10) @ _pow(Ms, 0.5)
    return A, G, Ms.A, Ns.A, ref


@pytest.mark.parametrize("m,n", [(300, 200), (200, 300)])
@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_weighted_moore_penrose(handle, m, n, prec):
    A, G, M, N, ref = weighted_problem(m, n, 150, seed=41)
    a = H.alpha_general(A, G)
    oref, _ = H.solve(A, H.x0_general(G, a), tol=1e-12, alpha=a, finish="outer")
    X, info = handle.solve(dev(A), kind="outer_g", G=dev(G), alpha=0.0, tol=1e-12, prec=prec, finish="clean")
    assert info["status"] == 0
    assert abs(info["alpha"] - a) <= 1e-12 * a
    X = host(X)
    assert rel(X, ref) < 1e-9 and rel(X, oref) < 1e-9
    MAX, NXA = M @ A @ X, N @ X @ A
    assert rel(A @ X @ A, A) < 1e-9 and rel(X @ A @ X, X) < 1e-9
    assert rel(MAX.T, MAX) < 1e-9 and rel(NXA.T, NXA) < 1e-9


def test_weighted_moore_penrose_complex(handle):
    A, G, M, N, ref = weighted_problem(120, 80, 60, seed=43, complex_=True)
    a = H.alpha_general(A, G)
    X, info = handle.solve_complex(dev(A), kind="outer_g", G=dev(G), alpha=0.0, tol=1e-12, prec="fp64_tc",
                                   finish="clean")
    assert info["status"] == 0
    assert abs(info["alpha"] - a) <= 1e-12 * a
    assert rel(host(X), ref) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_bott_duffin(handle, prec):
    s = W.spd(300, 0.01, 1.0, seed=44)
    P, Q = W.subspace_projector(300, 180, seed=45)
    ref = P @ np.linalg.inv(s.A @ P + (np.eye(300) - P))
    a = H.alpha_general(s.A, P)
    oref, _ = H.solve(s.A, H.x0_general(P, a), tol=1e-12, alpha=a, finish="outer")
    X, info = handle.solve(dev(s.A), kind="outer_g", G=dev(P), alpha=0.0, tol=1e-12, prec=prec, finish="clean")
    assert info["status"] == 0
    assert abs(info["alpha"] - a) <= 1e-12 * a
    assert rel(host(X), ref) < 1e-11 and rel(host(X), oref) < 1e-11


def test_batched_general_g_equals_single_solves(handle):
    """The group path takes the same alpha recipe per instance (on the padded
    slab) and the same X A X finish: each result equals the lone solve."""
    from paper_1604_07893_gb300._lib import Desc, Info
    probs = [weighted_problem(m, n, r, seed=50 + i) for i, (m, n, r) in
             enumerate([(130, 90, 70), (120, 100, 60), (90, 140, 80), (64, 40, 40)])]
    As = [dev(p[0]) for p in probs]
    Gs = [dev(p[1]) for p in probs]
    Xs = [torch.empty(p[0].shape[1], p[0].shape[0], dtype=torch.float64, device="cuda") for p in probs]
    kw = dict(kind="outer_g", alpha=0.0, tol=1e-12, prec="fp64_tc", finish="clean")
    descs = (Desc * len(probs))(*[handle.make_desc(A, X, G=G, **kw) for A, X, G in zip(As, Xs, Gs)])
    infos = (Info * len(probs))()
    rc = handle._lib.pinv_solve_batched(handle._h, len(probs), descs, C.c_void_p(0), infos)
    torch.cuda.synchronize()
    assert rc == 0
    for p, A, G, Xb, ib in zip(probs, As, Gs, Xs, infos):
        X1, i1 = handle.solve(A, G=G, **kw)
        assert abs(ib.alpha - i1["alpha"]) <= 1e-12 * i1["alpha"]
        assert rel(host(Xb), p[4]) < 1e-9
        assert rel(host(Xb), host(X1)) < 1e-10


def test_identity_g_alpha_recipe_on_a_positive_definite_matrix(handle):
    """G = I, A positive definite with lambda_max = 0.5: the Moore-Penrose recipe
    1/(||A||_1 ||A||_inf) would give alpha ~ 4 = 2/lambda_max (the top
    eigenvalue of I - alpha A at -1); the general-G recipe bounds lambda_max."""
    s = W.spd(200, 1e-2, 0.5, seed=46)
    X, info = handle.solve(dev(s.A), kind="outer_g", G=dev(np.eye(200)), alpha=0.0, tol=1e-12)
    assert info["status"] == 0
    assert info["alpha"] * 0.5 <= 1.0 + 1e-12
    assert rel(host(X), np.linalg.inv(s.A)) < 1e-11
