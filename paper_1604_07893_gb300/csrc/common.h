// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace pinv {

// One output of a fused GEMM epilogue:
//   out[i][j] = a_acc * acc[i][j] + a_s1 * s1[i][j] + a_s2 * s2[i][j] + (i == j ? a_id : 0)
// `out` may be null (nothing stored; useful when only the norms are wanted).
struct EpiTerm {
    double* out;
    int ld;
    double a_acc, a_s1, a_s2, a_id;
};

// Fused epilogue of a GEMM C = op(A) op(B): up to three outputs built from the
// accumulator, two side inputs of C's shape and the identity.  When `partials`
// is set, every CTA writes two FP64 partial sums in CTA order:
//   partials[2*cta]   = sum (out0 - s1)^2      (||X_{k+1} - X_k||_F^2 when s1 = X_k)
//   partials[2*cta+1] = sum s1^2               (||X_k||_F^2)
struct Epilogue {
    const double* s1; int ld1;
    const double* s2; int ld2;
    EpiTerm o[3];
    int nout;
    double* partials;
};

// The terms an epilogue output has, as integer flags computed on the host, so
// that the kernels test no FP64 value (on GB300 every FP64 instruction -- a
// compare included -- holds a sub-partition's FP64 unit for about 64 clocks
// per warp): OUT_NEG / OUT_MUL for a_acc = -1 / other than +-1.
enum { OUT_STORE = 1, OUT_NEG = 2, OUT_MUL = 4, OUT_S1 = 8, OUT_S2 = 16, OUT_ID = 32 };
inline int out_kind(const Epilogue& e, int o) {
    if (o >= e.nout) return 0;
    const EpiTerm& t = e.o[o];
    int k = 0;
    if (t.out) k |= OUT_STORE;
    if (t.a_acc == -1.0) k |= OUT_NEG;
    else if (t.a_acc != 1.0) k |= OUT_MUL;
    if (t.a_s1 != 0.0 && e.s1) k |= OUT_S1;
    if (t.a_s2 != 0.0 && e.s2) k |= OUT_S2;
    if (t.a_id != 0.0) k |= OUT_ID;
    return k;
}

#ifdef __CUDACC__
// FP64 arithmetic for the epilogues' terms, as volatile inline assembly so that
// the compiler does not evaluate it ahead of the uniform test of the term's
// flag (evaluating every term of every element and selecting had cost about
// four FP64 instructions per element at ~64 clocks per warp each).
__device__ __forceinline__ double dfma_keep(double a, double b, double c) {
    double d;
    asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(a), "d"(b), "d"(c));
    return d;
}
__device__ __forceinline__ double dmul_keep(double a, double b) {
    double d;
    asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(d) : "d"(a), "d"(b));
    return d;
}
__device__ __forceinline__ double dadd_keep(double a, double b) {
    double d;
    asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(d) : "d"(a), "d"(b));
    return d;
}
// -x by flipping the sign bit (integer pipe)
__device__ __forceinline__ double neg(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}
#endif

inline Epilogue epi_none() {
    Epilogue e{};
    e.nout = 0;
    return e;
}

// C (M x N) = op(A) (M x K) * op(B) (K x N), all row-major FP64.
// transA: A is stored K x M (element (i,k) at A[k*lda + i]); likewise transB.
// batch > 1: instance b uses every matrix (operands, side inputs, outputs) at
// +b*stride elements and writes its pair partials after those of instance b-1.
// sym_out (M == N, no partials): the product is known to be symmetric; only
// tiles on or above the diagonal are computed, off-diagonal ones also written
// transposed.
// tile: the CTA tile edge, 64, 32, 16 or 8 (gemm_f64_pick_tile chooses).
// Returns the pair partials per instance (the CTA count) or -1 on a launch error.
int gemm_f64(int M, int N, int K, const double* A, int lda, bool transA,
             const double* B, int ldb, bool transB, const Epilogue& epi, cudaStream_t st,
             int batch = 1, long long stride = 0, bool sym_out = false, int tile = 64);
int gemm_f64_ctas(int M, int N, int tile);
// The largest tile whose grid (times the batch) still covers `sms` CTAs, else 8.
int gemm_f64_pick_tile(int M, int N, int batch, int sms);
// Pair partials a product may need per instance, over every engine and tile:
// at most 64 per 64 x 64 block of the output (the 8 x 8 DMMA tile).
inline size_t partial_pairs_bound(size_t rows, size_t cols) { return 64 * ((rows + 63) / 64) * ((cols + 63) / 64); }

// Deterministic sum of `count` (pair) partials into out[0..1] (device); with
// batch > 1, instance b sums partials[2*count*b ...] into out[2b], out[2b+1].
void reduce_pairs(const double* partials, int count, double* out, cudaStream_t st, int batch = 1);

// Y (n x m, ldy) = alpha * A^T, A m x n (lda).
void transpose_scale(int m, int n, const double* A, int lda, double alpha, double* Y, int ldy,
                     cudaStream_t st);
// Y = alpha * X (rows x cols).
void scale_copy(int rows, int cols, const double* X, int ldx, double alpha, double* Y, int ldy,
                cudaStream_t st);
// out[0] = max column abs sum (||A||_1), out[1] = max row abs sum (||A||_inf).
void norms_1_inf(int m, int n, const double* A, int lda, double* out, double* scratch,
                 cudaStream_t st);
// out[0] = sum_ij P[i][j] * Q[j][i]  (trace of P Q), n x n.
void trace_of_product(int n, const double* P, int ldp, const double* Q, int ldq, double* out,
                      double* scratch, cudaStream_t st);
// out[0] = sum (P - Q)^2, out[1] = sum P^2 (Q may be P^T when `transQ`).
void diff_norms(int rows, int cols, const double* P, int ldp, const double* Q, int ldq,
                bool transQ, double* out, double* scratch, cudaStream_t st);
int diff_norms_scratch_pairs();

// Complex matrices as real embeddings E(Z) = [[Re Z, -Im Z], [Im Z, Re Z]]; Z is
// stored interleaved (re, im) with its leading dimension in complex elements.
// E (2m x 2n, lde) = E(Z), Z m x n.
void complex_embed(int m, int n, const double* Z, int ldz, double* E, int lde, cudaStream_t st);
// Z (r x c) from the left column half of E (2r x 2c): Z_ij = E[i][j] + i E[r+i][j].
void complex_extract(int r, int c, const double* E, int lde, double* Z, int ldz, cudaStream_t st);
// Right column half of an embedding (M rows, 2 N2 columns) from its left half.
void embed_mirror(int M, int N2, double* E, int ld, cudaStream_t st);
// out[0] = ||Z||_1, out[1] = ||Z||_inf with complex moduli, Z m x n read from E(Z).
void complex_norms_1_inf(int m, int n, const double* E, int lde, double* out, double* scratch, cudaStream_t st);

// X0 = alpha diag(1/a_ii) (Eq. choice3) into X (zero elsewhere already); with
// cplx, A and X are 2n x 2n embeddings of complex n x n matrices.
// out[0] (device) = the number of zero diagonal entries.
void jacobi_x0(int n, const double* A, int lda, double alpha, double* X, int ldx, bool cplx, double* out,
               cudaStream_t st);
// X[i][j] = 0 where |X[i][j]| < eps.
void chop(int rows, int cols, double* X, int ld, double eps, cudaStream_t st);

// X[i][j] = a deterministic pseudo-random value in (-1, 1) from (i, j, seed).
void fill_pattern(int rows, int cols, double* X, int ld, unsigned seed, cudaStream_t st);

// One instance of a batch: a caller matrix (rows x cols, leading dimension ld).
struct InstanceRef {
    const double* src;
    double* dst;
    int rows, cols, ld;
    int pad;
};
// slab_b (rows_pad x cols_pad, ld cols_pad, at slab0 + b*stride) = the
// instance's src, zero outside it; `table` is device memory.
void gather_pad(const InstanceRef* table, int batch, int rows_pad, int cols_pad, double* slab0,
                long long stride, cudaStream_t st);
// dst_b (rows_b x cols_b, ld_b) = the top-left block of slab_b (ld ld_slab) for
// every b with mask[b] != 0 (mask may be null: all); `table` is device memory.
void scatter_out(const InstanceRef* table, const int* mask, int batch, int rows_pad, int cols_pad,
                 const double* slab0, int ld_slab, long long stride, cudaStream_t st);
// slab_b = dst_b (the reverse of scatter_out, zero outside), for mask[b] != 0.
void scatter_in(const InstanceRef* table, const int* mask, int batch, int rows_pad, int cols_pad,
                double* slab0, int ld_slab, long long stride, cudaStream_t st);
// Y_b (n x m) = alpha[b] * A_b^T for every instance (alpha: device array).
void transpose_scale_batched(int m, int n, const double* A0, int lda, const double* alpha, double* Y0,
                             int ldy, long long stride, int batch, cudaStream_t st);
// Y_b = alpha[b] * X_b.
void scale_copy_batched(int rows, int cols, const double* X0, int ldx, const double* alpha, double* Y0,
                        int ldy, long long stride, int batch, cudaStream_t st);

}  // namespace pinv
