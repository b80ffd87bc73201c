// Mixed-precision loop engine: the seven products of Eq. PM on the tensor
// cores (tcgen05, operands staged by TMA, accumulators in TMEM).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace pinv {

struct MixedEngine;

struct MixedSchedule {
    int m, n, left;
    int prec;            // requested pinv_prec
    int bf16_loops;      // loops allowed in BF16 before the FP32-class loops
};

MixedEngine* mixed_create();
void mixed_destroy(MixedEngine*);
size_t mixed_workspace_bytes(int m, int n);
// Prepare operand shadows of A for a solve; fills the schedule.
int mixed_begin(MixedEngine*, int m, int n, int left, const double* A, int lda, int prec,
                cudaStream_t st, MixedSchedule* sched);
// Precision of loop k: 0 FP64, 1 BF16, 3 FP32-class.
int mixed_loop_precision(const MixedSchedule*, int k, double prev_step);
// One loop of Eq. PM from Xin to Xout (FP64 n x m, ld m) with products in
// precision `p`; the update X + D X is accumulated in FP64.  Writes pair
// partials for ||Xout - Xin||, ||Xin|| and returns their count (< 0 on error).
int mixed_pm_loop(MixedEngine*, const MixedSchedule*, int p, const double* Xin, double* Xout,
                  double* partials, cudaStream_t st);

// Kernel launches issued by the last mixed_pm_loop call.
int mixed_last_kernels(const MixedEngine*);

}  // namespace pinv
