"""Time one product of the GEMM engine through pinv_gemm.

  python -m paper_1604_07893_gb300.gemm_bench --M 3072 --N 3072 --K 4096 --prec fp64_tc

Prints the FP64-equivalent rate (2MNK / time) and the rate of BF16 tensor-core
work executed (2MNK x slice products / time), timed with CUDA events on the
launching stream after warm-up; inputs are larger than L2 at the default size.
"""

import argparse
import json

import numpy as np
import torch

from . import Handle

PAIRS = {"fp64_tc": 28, "fp32": 10, "mixed_bf16": 1, "fp64": None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=3072)
    ap.add_argument("--N", type=int, default=3072)
    ap.add_argument("--K", type=int, default=4096)
    ap.add_argument("--prec", default="fp64_tc", choices=list(PAIRS))
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(a.M, a.K, dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(a.K, a.N, dtype=torch.float64, device="cuda", generator=g)
    C = torch.empty(a.M, a.N, dtype=torch.float64, device="cuda")
    h = Handle(0)
    for _ in range(a.warmup):
        h.gemm(A, B, prec=a.prec, C=C)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        h.gemm(A, B, prec=a.prec, C=C)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flops = 2.0 * a.M * a.N * a.K
    ref = (A[:64].cpu().numpy() @ B.cpu().numpy())
    err = float(np.abs(C[:64].cpu().numpy() - ref).max() / np.abs(ref).max())
    out = {"M": a.M, "N": a.N, "K": a.K, "prec": a.prec, "ms_per_call": ms,
           "fp64_equivalent_tflops": flops / ms / 1e9,
           "tensor_tflops": flops * PAIRS[a.prec] / ms / 1e9 if PAIRS[a.prec] else None,
           "max_rel_err_rows64": err}
    print(json.dumps(out))
    h.close()


if __name__ == "__main__":
    main()
