// Tensor-core GEMM engine (tcgen05 + TMA + TMEM) for sm_103a.
#pragma once

#include <cstddef>

#include "common.h"

namespace pinv {

// Product precisions of the engine (values match pinv_prec where they overlap).
enum { TC_BF16 = 1, TC_FP32 = 3, TC_FP64 = 4 };

// S slices per operand, slice pairs with s + t <= L, exact = power-of-two grid
// slices (FP64/FP32-class) instead of one round-to-nearest BF16 slice.
struct TcMode {
    int S, L, exact;
};

TcMode tc_mode(int prec);
int tc_pairs(const TcMode& m);
size_t tc_workspace_bytes(int M, int N, int K, const TcMode& m, int batch = 1);
size_t tc_smem_bytes();

// C = op(A) op(B) with the fused FP64 epilogue `epi`.  `ws` holds the slices.
// ev_begin/ev_end (optional) are recorded around the tensor-core kernel alone.
// `err` is a device int that records a timed-out wait (0 = ok).  Adds the
// number of kernels launched to *kernels.  batch > 1: instance b uses every
// FP64 matrix (operands, side inputs, outputs) at +b*stride elements.  Returns
// the count of pair partials per instance (8 per 128 x 128 output tile, the
// instances one after another) or -1.  sym_out (M == N, no partials): the
// caller guarantees op(A) op(B) is symmetric; only the upper-triangle tiles are
// computed and each off-diagonal tile is also written transposed.
// wait_limit: polls before a wait of the kernel's main loop gives up (0: the
// default, about a second); the drain before exit always uses the default.
int tc_gemm(int M, int N, int K, const double* A, int lda, bool transA, const double* B, int ldb,
            bool transB, const Epilogue& epi, const TcMode& mode, void* ws, size_t ws_bytes, int* err,
            cudaStream_t st, int* kernels, cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr,
            int batch = 1, long long stride = 0, bool one_tile_per_cta = false,
            bool sym_out = false, unsigned wait_limit = 0);

}  // namespace pinv
