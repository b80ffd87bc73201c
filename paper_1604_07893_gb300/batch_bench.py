"""Time pinv_solve_batched on the uneven batch family.

  python -m paper_1604_07893_gb300.batch_bench --count 1024 --reps 2

m ~ U{32..512}, n ~ U{16..m}, rank n, singular values log-uniform in
[1e-3, 1] (Householder-product factors), alpha = 1/s_1^2, BF16 growth loops
then FP32-class loops and an FP32-class finish (PINV_PREC_BF16_FP32), the
order-18 stop at 0.25 (`--stop rel_fro`: the relative-step stop at 1e-6):
the settings of the batched workload line.  Prints, per call, the wall time
around the call (device synchronised on both sides), the tensor-core work the
instances' products executed and the loop counts.
"""

import argparse
import ctypes as C
import json
import time

import torch

from . import Handle, workloads as W
from ._lib import Desc, Info


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--stop", default="order18", choices=["order18", "rel_fro"])
    ap.add_argument("--tol", type=float, default=None, help="default: 0.25 (order18), 1e-6 (rel_fro)")
    a = ap.parse_args()
    ws = W.uneven_batch_fast(a.count, seed=a.seed)
    As = [torch.from_numpy(w.A).cuda() for w in ws]
    Xs = [torch.empty(w.A.shape[1], w.A.shape[0], dtype=torch.float64, device="cuda") for w in ws]
    h = Handle(0)
    st = torch.cuda.current_stream()
    for r in range(a.reps):
        tol = a.tol if a.tol is not None else (0.25 if a.stop == "order18" else 1e-6)
        descs = (Desc * a.count)(*[h.make_desc(A, X, alpha=1.0 / w.s[0] ** 2, tol=tol, stop=a.stop,
                                               prec="bf16_fp32", finish="clean") for A, X, w in zip(As, Xs, ws)])
        infos = (Info * a.count)()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = h._lib.pinv_solve_batched(h._h, a.count, descs, C.c_void_p(st.cuda_stream), infos)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        iters = [infos[i].iters for i in range(a.count)]
        print(json.dumps({"rep": r, "status": rc, "count": a.count, "ms": t * 1e3,
                          "tensor_flops": sum(infos[i].tensor_flops for i in range(a.count)),
                          "loops": [min(iters), max(iters)]}), flush=True)
        if rc != 0:
            raise SystemExit(1)
    h.close()


if __name__ == "__main__":
    main()
