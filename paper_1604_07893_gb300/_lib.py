"""ctypes binding of ``include/pinv.h``: argument marshalling only.

Every step of the computation runs in ``libpinv.so``; this module converts
torch tensors (device memory and streams) or numpy arrays (host buffers) into
the C structures and back.  If the library has not been built it raises: there
is no other code path.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpinv.so")

PINV_OK, PINV_PENDING = 0, 1
ERRORS = {-1: "PINV_ERR_ARG", -2: "PINV_ERR_BUDGET", -3: "PINV_ERR_NONFINITE", -4: "PINV_ERR_DIVERGED",
          -5: "PINV_ERR_MAXITER", -6: "PINV_ERR_TIMEOUT", -7: "PINV_ERR_CUDA", -8: "PINV_ERR_UNKNOWN_ID",
          -9: "PINV_ERR_BUSY"}
KIND = {"moore_penrose": 0, "drazin": 1, "outer_g": 2, "drazin_normal": 3}
STOP = {"rel_fro": 0, "paper": 1, "order18": 2}
PREC = {"fp64": 0, "mixed_bf16": 1, "mixed_fp8": 2, "fp32": 3, "fp64_tc": 4, "bf16_fp32": 5,
        "fp32_refine": 6}
VARIANT = {"plain": 0, "stabilized": 1}
FINISH = {None: 0, "none": 0, "clean": 1}
HISTORY = 128

EXPORTS = ("pinv_init", "pinv_destroy", "pinv_solve", "pinv_solve_complex", "pinv_preconditioner",
           "pinv_solve_batched", "pinv_submit",
           "pinv_poll", "pinv_alpha_estimate", "pinv_step", "pinv_gemm", "pinv_autotune", "pinv_drazin_index",
           "pinv_step_noalloc", "pinv_set_wait_limit", "pinv_serving_stats")
NOALLOC_MAX_DIM = 128


class Config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("device", C.c_int), ("max_queued", C.c_int),
                ("reserved", C.c_int * 5)]


class ServingStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("rejected", C.c_uint64), ("admitted", C.c_uint64),
                ("completed", C.c_uint64), ("queued", C.c_int), ("running", C.c_int), ("groups", C.c_int),
                ("reserved", C.c_int), ("device_bytes", C.c_size_t)]


class Desc(C.Structure):
    _fields_ = [("m", C.c_int), ("n", C.c_int),
                ("A", C.c_void_p), ("lda", C.c_int),
                ("X", C.c_void_p), ("ldx", C.c_int),
                ("G", C.c_void_p), ("ldg", C.c_int),
                ("kind", C.c_int), ("drazin_index", C.c_int),
                ("alpha", C.c_double), ("tol", C.c_double), ("stop", C.c_int),
                ("max_iter", C.c_int), ("prec", C.c_int), ("variant", C.c_int),
                ("switch_tol", C.c_double), ("finish", C.c_int), ("host_buffers", C.c_int),
                ("check", C.c_int), ("profile", C.c_int), ("symmetric", C.c_int),
                ("reserved", C.c_int * 2)]


class PrecondDesc(C.Structure):
    _fields_ = [("n", C.c_int), ("A", C.c_void_p), ("lda", C.c_int), ("X", C.c_void_p), ("ldx", C.c_int),
                ("loops", C.c_int), ("alpha", C.c_double), ("chop", C.c_double), ("prec", C.c_int),
                ("complex_matrix", C.c_int), ("host_buffers", C.c_int), ("profile", C.c_int),
                ("reserved", C.c_int * 4)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("loops_run", C.c_int),
                ("stabilized_loops", C.c_int), ("stop_reason", C.c_int), ("side", C.c_int),
                ("rel_step", C.c_double), ("alpha", C.c_double),
                ("penrose", C.c_double * 4), ("drazin", C.c_double * 3), ("ms", C.c_float),
                ("gemms", C.c_int), ("kernels", C.c_int), ("gemm_ms", C.c_float),
                ("gemm_flops", C.c_double), ("tensor_flops", C.c_double),
                ("history", C.c_double * HISTORY),
                ("precision", C.c_byte * HISTORY)]

    def to_dict(self) -> dict:
        n = min(self.loops_run, HISTORY)
        return dict(status=self.status, iters=self.iters, loops_run=self.loops_run,
                    stabilized_loops=self.stabilized_loops, stop_reason=self.stop_reason,
                    side="left" if self.side else "right", rel_step=self.rel_step, alpha=self.alpha,
                    penrose=list(self.penrose), drazin=list(self.drazin), ms=self.ms,
                    gemms=self.gemms, kernels=self.kernels, gemm_ms=self.gemm_ms,
                    gemm_flops=self.gemm_flops, tensor_flops=self.tensor_flops,
                    history=list(self.history[:n]),
                    precision=list(self.precision[:n]))


_lib = None


def load() -> C.CDLL:
    """Load libpinv.so (built in-tree by ``build.py``); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1604_07893_gb300.build.build() first")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    lib.pinv_init.argtypes = [P(C.c_void_p), P(Config)]
    lib.pinv_destroy.argtypes = [C.c_void_p]
    lib.pinv_destroy.restype = None
    lib.pinv_solve.argtypes = [C.c_void_p, P(Desc), C.c_void_p, P(Info)]
    lib.pinv_solve_complex.argtypes = [C.c_void_p, P(Desc), C.c_void_p, P(Info)]
    lib.pinv_preconditioner.argtypes = [C.c_void_p, P(PrecondDesc), C.c_void_p, P(Info)]
    lib.pinv_solve_batched.argtypes = [C.c_void_p, C.c_int, P(Desc), C.c_void_p, P(Info)]
    lib.pinv_submit.argtypes = [C.c_void_p, P(Desc), P(C.c_uint64)]
    lib.pinv_poll.argtypes = [C.c_void_p, C.c_uint64, P(Info)]
    lib.pinv_alpha_estimate.argtypes = [C.c_void_p, P(Desc), C.c_void_p, P(C.c_double)]
    lib.pinv_step.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                              C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, P(C.c_double)]
    lib.pinv_gemm.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
                              C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    lib.pinv_autotune.argtypes = [C.c_void_p, C.c_void_p, P(C.c_int)]
    lib.pinv_drazin_index.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p, P(C.c_int),
                                      P(C.c_int)]
    lib.pinv_step_noalloc.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                      C.c_void_p, C.c_int, C.c_int, C.c_void_p, P(C.c_double)]
    lib.pinv_set_wait_limit.argtypes = [C.c_void_p, C.c_uint]
    lib.pinv_serving_stats.argtypes = [C.c_void_p, P(ServingStats)]
    for name in EXPORTS:
        if name != "pinv_destroy":
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class PinvError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}")
        self.code = code


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _dev_ptr(t, cplx: bool = False) -> int:
    import torch
    want = torch.complex128 if cplx else torch.float64
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want):
        raise TypeError(f"expected a CUDA {want} tensor")
    if t.stride(1) != 1:
        raise ValueError("matrices must be row-major (unit column stride)")
    return t.data_ptr()


class Handle:
    """pinv_init / pinv_destroy."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_queued: int = 0):
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        cfg = Config(hbm_budget_bytes=hbm_budget_bytes, device=device, max_queued=max_queued)
        rc = lib.pinv_init(C.byref(self._h), C.byref(cfg))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_init")

    def close(self):
        if self._h:
            self._lib.pinv_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- helpers
    @staticmethod
    def make_desc(A, X, *, kind="moore_penrose", G=None, drazin_index=0, alpha=0.0, tol=1e-12,
                  stop="rel_fro", max_iter=0, prec="fp64", variant="plain", switch_tol=0.0,
                  finish=None, check=False, host=False, profile=False, symmetric=False,
                  cplx=False) -> Desc:
        if host:
            import numpy as np
            want = np.complex128 if cplx else np.float64
            for M in (A, X) + ((G,) if G is not None else ()):
                if not (isinstance(M, np.ndarray) and M.dtype == want and M.flags.c_contiguous):
                    raise TypeError(f"host buffers must be C-contiguous {np.dtype(want)} numpy arrays")
            a_ptr, x_ptr = A.ctypes.data, X.ctypes.data
            g_ptr = G.ctypes.data if G is not None else None
            lda, ldx, ldg = A.shape[1], X.shape[1], (G.shape[1] if G is not None else 0)
        else:
            a_ptr, x_ptr = _dev_ptr(A, cplx), _dev_ptr(X, cplx)
            g_ptr = _dev_ptr(G, cplx) if G is not None else None
            lda, ldx = A.stride(0), X.stride(0)
            ldg = G.stride(0) if G is not None else 0
        m, n = A.shape
        if tuple(X.shape) != (n, m):
            raise ValueError("X must be n x m")
        return Desc(m=m, n=n, A=a_ptr, lda=lda, X=x_ptr, ldx=ldx, G=g_ptr, ldg=ldg,
                    kind=KIND[kind], drazin_index=drazin_index, alpha=alpha, tol=tol,
                    stop=STOP[stop], max_iter=max_iter, prec=PREC[prec], variant=VARIANT[variant],
                    switch_tol=switch_tol, finish=FINISH[finish], host_buffers=1 if host else 0,
                    check=1 if check else 0, profile=1 if profile else 0,
                    symmetric=1 if symmetric else 0)

    # ------------------------------------------------------------ entry points
    def solve(self, A, X=None, *, stream=None, raise_on_error=True, **kw):
        """pinv_solve.  A: CUDA float64 tensor (or numpy with host=True).
        Returns (X, info dict)."""
        host = kw.get("host", False)
        if X is None:
            if host:
                import numpy as np
                X = np.empty((A.shape[1], A.shape[0]), dtype=np.float64)
            else:
                import torch
                X = torch.empty((A.shape[1], A.shape[0]), dtype=torch.float64, device=A.device)
        d = self.make_desc(A, X, **kw)
        info = Info()
        st = 0 if host and stream is None else _stream_ptr(stream)
        rc = self._lib.pinv_solve(self._h, C.byref(d), C.c_void_p(st), C.byref(info))
        if rc != PINV_OK and raise_on_error:
            raise PinvError(rc, "pinv_solve")
        return X, info.to_dict()

    def solve_complex(self, A, X=None, *, stream=None, raise_on_error=True, **kw):
        """pinv_solve_complex.  A: CUDA complex128 tensor (or complex128 numpy
        with host=True).  Returns (X, info dict)."""
        host = kw.get("host", False)
        if X is None:
            if host:
                import numpy as np
                X = np.empty((A.shape[1], A.shape[0]), dtype=np.complex128)
            else:
                import torch
                X = torch.empty((A.shape[1], A.shape[0]), dtype=torch.complex128, device=A.device)
        d = self.make_desc(A, X, cplx=True, **kw)
        info = Info()
        st = 0 if host and stream is None else _stream_ptr(stream)
        rc = self._lib.pinv_solve_complex(self._h, C.byref(d), C.c_void_p(st), C.byref(info))
        if rc != PINV_OK and raise_on_error:
            raise PinvError(rc, "pinv_solve_complex")
        return X, info.to_dict()

    def preconditioner(self, A, X=None, *, loops=1, chop=0.0, alpha=0.0, prec="fp64", host=False,
                       profile=False, stream=None, raise_on_error=True):
        """pinv_preconditioner: X_loops from the Jacobi X0 (Section 8, Example 3).
        A: square CUDA float64/complex128 tensor, or numpy with host=True.
        Returns (X, info dict)."""
        n = A.shape[0]
        if A.shape[1] != n:
            raise ValueError("square matrix required")
        if host:
            import numpy as np
            cplx = A.dtype == np.complex128
            if X is None:
                X = np.empty((n, n), dtype=A.dtype)
            for M in (A, X):
                if not (isinstance(M, np.ndarray) and M.dtype == A.dtype and M.flags.c_contiguous and
                        M.dtype in (np.float64, np.complex128)):
                    raise TypeError("host buffers must be C-contiguous float64 or complex128 numpy arrays")
            a_ptr, x_ptr, lda, ldx = A.ctypes.data, X.ctypes.data, A.shape[1], X.shape[1]
        else:
            import torch
            cplx = A.dtype == torch.complex128
            if X is None:
                X = torch.empty((n, n), dtype=A.dtype, device=A.device)
            a_ptr, x_ptr, lda, ldx = _dev_ptr(A, cplx), _dev_ptr(X, cplx), A.stride(0), X.stride(0)
        d = PrecondDesc(n=n, A=a_ptr, lda=lda, X=x_ptr, ldx=ldx, loops=loops, alpha=alpha, chop=chop,
                        prec=PREC[prec], complex_matrix=1 if cplx else 0, host_buffers=1 if host else 0,
                        profile=1 if profile else 0)
        info = Info()
        st = 0 if host and stream is None else _stream_ptr(stream)
        rc = self._lib.pinv_preconditioner(self._h, C.byref(d), C.c_void_p(st), C.byref(info))
        if rc != PINV_OK and raise_on_error:
            raise PinvError(rc, "pinv_preconditioner")
        return X, info.to_dict()

    def solve_batched(self, As, Xs=None, *, stream=None, **kw):
        import torch
        if Xs is None:
            Xs = [torch.empty((A.shape[1], A.shape[0]), dtype=torch.float64, device=A.device) for A in As]
        if not As:
            return [], []
        descs = (Desc * len(As))(*[self.make_desc(A, X, **kw) for A, X in zip(As, Xs)])
        infos = (Info * len(As))()
        rc = self._lib.pinv_solve_batched(self._h, len(As), descs, C.c_void_p(_stream_ptr(stream)), infos)
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_solve_batched")
        return Xs, [i.to_dict() for i in infos]

    def submit(self, A, X, **kw) -> int:
        """pinv_submit: queue a problem; A, X (and G) must stay alive until poll
        returns its final status."""
        d = self.make_desc(A, X, **kw)
        rid = C.c_uint64()
        rc = self._lib.pinv_submit(self._h, C.byref(d), C.byref(rid))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_submit")
        return rid.value

    def serving_stats(self) -> dict:
        """pinv_serving_stats: counters of the serving loop and its backlog."""
        st = ServingStats()
        rc = self._lib.pinv_serving_stats(self._h, C.byref(st))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_serving_stats")
        return {k: getattr(st, k) for k, _ in ServingStats._fields_ if k != "reserved"}

    def poll(self, rid: int):
        """Returns None while pending, else (status, info dict)."""
        info = Info()
        rc = self._lib.pinv_poll(self._h, C.c_uint64(rid), C.byref(info))
        if rc == PINV_PENDING:
            return None
        return rc, info.to_dict()

    def alpha_estimate(self, A, *, stream=None) -> float:
        import torch
        X = torch.empty((1, 1), dtype=torch.float64, device=A.device)
        d = Desc(m=A.shape[0], n=A.shape[1], A=_dev_ptr(A), lda=A.stride(0), X=X.data_ptr(), ldx=1)
        out = C.c_double()
        rc = self._lib.pinv_alpha_estimate(self._h, C.byref(d), C.c_void_p(_stream_ptr(stream)), C.byref(out))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_alpha_estimate")
        return out.value

    def gemm(self, A, B, *, trans_a=False, trans_b=False, prec="fp64", C=None, stream=None):
        """pinv_gemm: C = op(A) op(B) with the product engine of `prec`."""
        import torch
        M = A.shape[1] if trans_a else A.shape[0]
        K = A.shape[0] if trans_a else A.shape[1]
        N = B.shape[0] if trans_b else B.shape[1]
        if (B.shape[1] if trans_b else B.shape[0]) != K:
            raise ValueError("inner dimensions differ")
        if C is None:
            C = torch.empty((M, N), dtype=torch.float64, device=A.device)
        rc = self._lib.pinv_gemm(self._h, M, N, K, _dev_ptr(A),
                                 A.stride(0), 1 if trans_a else 0, _dev_ptr(B), B.stride(0),
                                 1 if trans_b else 0, _dev_ptr(C), C.stride(0), PREC[prec],
                                 _stream_ptr(stream))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_gemm")
        return C

    def set_wait_limit(self, polls: int):
        """pinv_set_wait_limit: polls before a tensor-core kernel wait gives up
        (0 = the default of about a second), for every later call."""
        rc = self._lib.pinv_set_wait_limit(self._h, C.c_uint(polls))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_set_wait_limit")

    def drazin_index(self, A, *, max_index: int = 16, stream=None):
        """pinv_drazin_index: ind(A) of a square device matrix and the ranks of
        A^0 .. A^(ind+1); raises PinvError if the index exceeds max_index."""
        n = A.shape[0]
        if A.shape[1] != n:
            raise ValueError("square matrix required")
        idx = C.c_int()
        ranks = (C.c_int * (max_index + 2))()
        rc = self._lib.pinv_drazin_index(self._h, n, C.c_void_p(_dev_ptr(A)), A.stride(0), max_index,
                                         C.c_void_p(_stream_ptr(stream)), C.byref(idx), ranks)
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_drazin_index")
        return idx.value, [ranks[k] for k in range(idx.value + 2)]

    def autotune(self, stream=None) -> int:
        """pinv_autotune: measure the DMMA / tensor-core crossover for FP64-class
        products on this device; returns the crossover size (0 = tensor cores
        everywhere)."""
        out = C.c_int()
        rc = self._lib.pinv_autotune(self._h, C.c_void_p(_stream_ptr(stream)), C.byref(out))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_autotune")
        return out.value

    def step(self, A, X_in, X_out=None, *, prec="fp64", stabilized=False, stream=None):
        """pinv_step: one loop of Eq. PM (or PM-modified).  Returns (X_out, rel_step)."""
        import torch
        if X_out is None:
            X_out = torch.empty_like(X_in)
        m, n = A.shape
        rel = C.c_double()
        rc = self._lib.pinv_step(self._h, m, n, C.c_void_p(_dev_ptr(A)), A.stride(0),
                                 C.c_void_p(_dev_ptr(X_in)), C.c_void_p(_dev_ptr(X_out)),
                                 X_in.stride(0), PREC[prec], 1 if stabilized else 0,
                                 C.c_void_p(_stream_ptr(stream)), C.byref(rel))
        if rc != PINV_OK:
            raise PinvError(rc, "pinv_step")
        return X_out, rel.value


def step_noalloc(A, X_in, X_out=None, *, stabilized=False, stream=None):
    """pinv_step_noalloc: one FP64 loop using the library's static scratch
    (no allocation inside the call; m, n <= 128).  Returns (X_out, rel_step)."""
    import torch
    lib = load()
    if X_out is None:
        X_out = torch.empty_like(X_in)
    m, n = A.shape
    rel = C.c_double()
    rc = lib.pinv_step_noalloc(m, n, C.c_void_p(_dev_ptr(A)), A.stride(0), C.c_void_p(_dev_ptr(X_in)),
                               C.c_void_p(_dev_ptr(X_out)), X_in.stride(0), 1 if stabilized else 0,
                               C.c_void_p(_stream_ptr(stream)), C.byref(rel))
    if rc != PINV_OK:
        raise PinvError(rc, "pinv_step_noalloc")
    return X_out, rel.value
