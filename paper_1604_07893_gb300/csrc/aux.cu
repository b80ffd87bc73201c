// Small FP64 kernels around the GEMMs: initial values (Section 4), the
// deterministic reduction of stop-norm partials, and residual norms.
//
// All reductions are two-level with a fixed CTA count and a fixed order, so a
// result is bitwise reproducible from run to run.

#include "common.h"

namespace pinv {
namespace {

constexpr int RED_CTAS = 256;     // fixed first-level width of every reduction
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, sh[w]);
    __syncthreads();
    return s;
}

__global__ void reduce_pairs_kernel(const double* p, int count, double* out) {
    __shared__ double sh[32];
    p += 2LL * count * blockIdx.x;   // instance blockIdx.x of a batch
    out += 2 * blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        a += p[2 * i];
        b += p[2 * i + 1];
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
}

__global__ void transpose_scale_kernel(int m, int n, const double* A, int lda, double alpha,
                                       double* Y, int ldy) {
    __shared__ double t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // bx over n (cols of A), by over m
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int i = by + r, j = bx + threadIdx.x;
        if (i < m && j < n) t[r][threadIdx.x] = A[(size_t)i * lda + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int j = bx + r, i = by + threadIdx.x;   // Y[j][i] = alpha * A[i][j]
        if (i < m && j < n) Y[(size_t)j * ldy + i] = alpha * t[threadIdx.x][r];
    }
}

__global__ void scale_copy_kernel(int rows, int cols, const double* X, int ldx, double alpha,
                                  double* Y, int ldy) {
    size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t i = e / cols, j = e % cols;
        Y[i * ldy + j] = alpha * X[i * ldx + j];
    }
}

// Partial column sums (block handles a strip of columns over all rows) and row sums.
__global__ void row_abs_max_kernel(int m, int n, const double* A, int lda, double* part) {
    __shared__ double sh[32];
    double best = 0.0;
    for (int i = blockIdx.x; i < m; i += gridDim.x) {
        double s = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) s += fabs(A[(size_t)i * lda + j]);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) best = fmax(best, s);
    }
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

__global__ void col_abs_max_kernel(int m, int n, const double* A, int lda, double* part) {
    __shared__ double sh[32];
    double best = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += fabs(A[(size_t)i * lda + j]);
        best = fmax(best, s);
    }
    best = block_max(best, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

__global__ void max_kernel(const double* part, int count, double* out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v = fmax(v, part[i]);
    v = block_max(v, sh);
    if (threadIdx.x == 0) *out = v;
}

__global__ void trace_product_kernel(int n, const double* P, int ldp, const double* Q, int ldq,
                                     double* part) {
    __shared__ double sh[32];
    double s = 0.0;
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t i = e / n, j = e % n;
        s += P[i * ldp + j] * Q[j * ldq + i];
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = s, part[2 * blockIdx.x + 1] = 0.0;
}

__global__ void diff_norms_kernel(int rows, int cols, const double* P, int ldp, const double* Q,
                                  int ldq, int transQ, double* part) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t i = e / cols, j = e % cols;
        double p = P[i * ldp + j];
        double q = transQ ? Q[j * ldq + i] : Q[i * ldq + j];
        a += (p - q) * (p - q);
        b += p * p;
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = a, part[2 * blockIdx.x + 1] = b;
}

__global__ void gather_pad_kernel(const InstanceRef* table, int rows_pad, int cols_pad, double* slab0,
                                  long long stride) {
    const InstanceRef r = table[blockIdx.z];
    double* dst = slab0 + (long long)blockIdx.z * stride;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols_pad; j += gridDim.x * blockDim.x) {
        if (i < rows_pad)
            dst[(size_t)i * cols_pad + j] = (i < r.rows && j < r.cols) ? r.src[(size_t)i * r.ld + j] : 0.0;
    }
}

__global__ void scatter_kernel(const InstanceRef* table, const int* mask, int rows_pad, int cols_pad,
                               double* slab0, int ld_slab, long long stride, int to_caller) {
    if (mask && !mask[blockIdx.z]) return;
    const InstanceRef r = table[blockIdx.z];
    double* slab = slab0 + (long long)blockIdx.z * stride;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= rows_pad) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols_pad; j += gridDim.x * blockDim.x) {
        const bool inside = i < r.rows && j < r.cols;
        if (to_caller) {
            if (inside) r.dst[(size_t)i * r.ld + j] = slab[(size_t)i * ld_slab + j];
        } else {
            slab[(size_t)i * ld_slab + j] = inside ? r.dst[(size_t)i * r.ld + j] : 0.0;
        }
    }
}

__global__ void transpose_scale_batched_kernel(int m, int n, const double* A0, int lda, const double* alpha,
                                               double* Y0, int ldy, long long stride) {
    __shared__ double t[32][33];
    const double* A = A0 + (long long)blockIdx.z * stride;
    double* Y = Y0 + (long long)blockIdx.z * stride;
    const double a = alpha[blockIdx.z];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int i = by + r, j = bx + threadIdx.x;
        if (i < m && j < n) t[r][threadIdx.x] = A[(size_t)i * lda + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int j = bx + r, i = by + threadIdx.x;
        if (i < m && j < n) Y[(size_t)j * ldy + i] = a * t[threadIdx.x][r];
    }
}

__global__ void scale_copy_batched_kernel(int rows, int cols, const double* X0, int ldx, const double* alpha,
                                          double* Y0, int ldy, long long stride) {
    const double* X = X0 + (long long)blockIdx.z * stride;
    double* Y = Y0 + (long long)blockIdx.z * stride;
    const double a = alpha[blockIdx.z];
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= rows) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += gridDim.x * blockDim.x)
        Y[(size_t)i * ldy + j] = a * X[(size_t)i * ldx + j];
}

__global__ void fill_pattern_kernel(int rows, int cols, double* X, int ld, unsigned seed) {
    const size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)e * 2654435761u ^ seed * 40503u;
        h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
        X[(e / cols) * ld + e % cols] = ((double)h / 4294967296.0) * 2.0 - 1.0;
    }
}

// ---- complex matrices as real embeddings E(Z) = [[Re Z, -Im Z], [Im Z, Re Z]]
// (E is a *-homomorphism: E(ZW) = E(Z)E(W), E(Z^*) = E(Z)^T, so every
// generalized inverse of Z is read off the same inverse of E(Z)).

// E (2m x 2n, lde) from Z (m x n complex, interleaved re/im, ldz complex elements).
__global__ void complex_embed_kernel(int m, int n, const double* Z, int ldz, double* E, int lde) {
    const size_t total = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / n, j = e % n;
        const double re = Z[2 * (i * ldz + j)], im = Z[2 * (i * ldz + j) + 1];
        E[i * lde + j] = re;
        E[i * lde + n + j] = -im;
        E[(i + m) * lde + j] = im;
        E[(i + m) * lde + n + j] = re;
    }
}

// Z (r x c complex, ldz) = the left column half of E (2r x 2c, lde): (E[i][j], E[r+i][j]).
__global__ void complex_extract_kernel(int r, int c, const double* E, int lde, double* Z, int ldz) {
    const size_t total = (size_t)r * c;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / c, j = e % c;
        Z[2 * (i * ldz + j)] = E[i * lde + j];
        Z[2 * (i * ldz + j) + 1] = E[(i + r) * lde + j];
    }
}

// Right column half of an embedding from its left half [Re; Im] (M = 2r rows,
// N2 = c columns): E[i][c+j] = -E[r+i][j], E[r+i][c+j] = E[i][j].
__global__ void embed_mirror_kernel(int M, int N2, double* E, int ld) {
    const int r = M / 2;
    const size_t total = (size_t)r * N2;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / N2, j = e % N2;
        const double re = E[i * ld + j], im = E[(i + r) * ld + j];
        E[i * ld + N2 + j] = -im;
        E[(i + r) * ld + N2 + j] = re;
    }
}

// ||Z||_1 and ||Z||_inf partials with |z_ij| = hypot(Re, Im) read from the
// left half of E (Z is m x n, E 2m x 2n).
__global__ void complex_row_abs_max_kernel(int m, int n, const double* E, int lde, double* part) {
    __shared__ double sh[32];
    double best = 0.0;
    for (int i = blockIdx.x; i < m; i += gridDim.x) {
        double s = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            s += hypot(E[(size_t)i * lde + j], E[(size_t)(i + m) * lde + j]);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) best = fmax(best, s);
    }
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

__global__ void complex_col_abs_max_kernel(int m, int n, const double* E, int lde, double* part) {
    __shared__ double sh[32];
    double best = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += hypot(E[(size_t)i * lde + j], E[(size_t)(i + m) * lde + j]);
        best = fmax(best, s);
    }
    best = block_max(best, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

// X0 = alpha diag(1/a_11, ..., 1/a_nn) (Eq. choice3) into X, zeroed by the
// caller.  cplx: A and X are embeddings (2n x 2n) of complex n x n matrices,
// a_i = E[i][i] + i E[n+i][i] and 1/a_i = conj(a_i)/|a_i|^2.  One CTA;
// out[0] = the number of zero diagonal entries (left unwritten in X).
__global__ void jacobi_x0_kernel(int n, const double* A, int lda, double alpha, double* X, int ldx, int cplx,
                                 double* out) {
    __shared__ int zeros;
    if (threadIdx.x == 0) zeros = 0;
    __syncthreads();
    int local = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (!cplx) {
            const double a = A[(size_t)i * lda + i];
            if (a == 0.0) { ++local; continue; }
            X[(size_t)i * ldx + i] = alpha / a;
        } else {
            const double re = A[(size_t)i * lda + i], im = A[(size_t)(i + n) * lda + i];
            const double d = re * re + im * im;
            if (d == 0.0) { ++local; continue; }
            const double xr = alpha * re / d, xi = -alpha * im / d;
            X[(size_t)i * ldx + i] = xr;
            X[(size_t)i * ldx + n + i] = -xi;
            X[(size_t)(i + n) * ldx + i] = xi;
            X[(size_t)(i + n) * ldx + n + i] = xr;
        }
    }
    if (local) atomicAdd(&zeros, local);
    __syncthreads();
    if (threadIdx.x == 0) out[0] = (double)zeros;
}

// Entries of magnitude below eps set to 0 (on an embedding each entry is one
// real or imaginary part, so complex parts are chopped separately).
__global__ void chop_kernel(int rows, int cols, double* X, int ld, double eps) {
    const size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        double* p = X + (e / cols) * ld + e % cols;
        if (fabs(*p) < eps) *p = 0.0;
    }
}

}  // namespace

void fill_pattern(int rows, int cols, double* X, int ld, unsigned seed, cudaStream_t st) {
    fill_pattern_kernel<<<152 * 4, 256, 0, st>>>(rows, cols, X, ld, seed);
}

void gather_pad(const InstanceRef* table, int batch, int rows_pad, int cols_pad, double* slab0,
                long long stride, cudaStream_t st) {
    dim3 blk(32, 8), grid((cols_pad + 31) / 32 < 8 ? (cols_pad + 31) / 32 : 8, (rows_pad + 7) / 8, batch);
    gather_pad_kernel<<<grid, blk, 0, st>>>(table, rows_pad, cols_pad, slab0, stride);
}

void scatter_out(const InstanceRef* table, const int* mask, int batch, int rows_pad, int cols_pad,
                 const double* slab0, int ld_slab, long long stride, cudaStream_t st) {
    dim3 blk(32, 8), grid((cols_pad + 31) / 32 < 8 ? (cols_pad + 31) / 32 : 8, (rows_pad + 7) / 8, batch);
    scatter_kernel<<<grid, blk, 0, st>>>(table, mask, rows_pad, cols_pad, const_cast<double*>(slab0), ld_slab,
                                         stride, 1);
}

void scatter_in(const InstanceRef* table, const int* mask, int batch, int rows_pad, int cols_pad,
                double* slab0, int ld_slab, long long stride, cudaStream_t st) {
    dim3 blk(32, 8), grid((cols_pad + 31) / 32 < 8 ? (cols_pad + 31) / 32 : 8, (rows_pad + 7) / 8, batch);
    scatter_kernel<<<grid, blk, 0, st>>>(table, mask, rows_pad, cols_pad, slab0, ld_slab, stride, 0);
}

void transpose_scale_batched(int m, int n, const double* A0, int lda, const double* alpha, double* Y0,
                             int ldy, long long stride, int batch, cudaStream_t st) {
    dim3 grid((n + 31) / 32, (m + 31) / 32, batch), block(32, 8);
    transpose_scale_batched_kernel<<<grid, block, 0, st>>>(m, n, A0, lda, alpha, Y0, ldy, stride);
}

void scale_copy_batched(int rows, int cols, const double* X0, int ldx, const double* alpha, double* Y0,
                        int ldy, long long stride, int batch, cudaStream_t st) {
    dim3 blk(32, 8), grid((cols + 31) / 32 < 8 ? (cols + 31) / 32 : 8, (rows + 7) / 8, batch);
    scale_copy_batched_kernel<<<grid, blk, 0, st>>>(rows, cols, X0, ldx, alpha, Y0, ldy, stride);
}

void reduce_pairs(const double* partials, int count, double* out, cudaStream_t st, int batch) {
    reduce_pairs_kernel<<<batch, RED_THREADS, 0, st>>>(partials, count, out);
}

void transpose_scale(int m, int n, const double* A, int lda, double alpha, double* Y, int ldy,
                     cudaStream_t st) {
    dim3 grid((n + 31) / 32, (m + 31) / 32), block(32, 8);
    transpose_scale_kernel<<<grid, block, 0, st>>>(m, n, A, lda, alpha, Y, ldy);
}

void scale_copy(int rows, int cols, const double* X, int ldx, double alpha, double* Y, int ldy,
                cudaStream_t st) {
    size_t total = (size_t)rows * cols;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    scale_copy_kernel<<<blocks, 256, 0, st>>>(rows, cols, X, ldx, alpha, Y, ldy);
}

void norms_1_inf(int m, int n, const double* A, int lda, double* out, double* scratch,
                 cudaStream_t st) {
    col_abs_max_kernel<<<RED_CTAS, RED_THREADS, 0, st>>>(m, n, A, lda, scratch);
    max_kernel<<<1, RED_THREADS, 0, st>>>(scratch, RED_CTAS, out);
    row_abs_max_kernel<<<RED_CTAS, RED_THREADS, 0, st>>>(m, n, A, lda, scratch + RED_CTAS);
    max_kernel<<<1, RED_THREADS, 0, st>>>(scratch + RED_CTAS, RED_CTAS, out + 1);
}

void trace_of_product(int n, const double* P, int ldp, const double* Q, int ldq, double* out,
                      double* scratch, cudaStream_t st) {
    trace_product_kernel<<<RED_CTAS, RED_THREADS, 0, st>>>(n, P, ldp, Q, ldq, scratch);
    reduce_pairs_kernel<<<1, RED_THREADS, 0, st>>>(scratch, RED_CTAS, out);
}

void diff_norms(int rows, int cols, const double* P, int ldp, const double* Q, int ldq,
                bool transQ, double* out, double* scratch, cudaStream_t st) {
    diff_norms_kernel<<<RED_CTAS, RED_THREADS, 0, st>>>(rows, cols, P, ldp, Q, ldq,
                                                        transQ ? 1 : 0, scratch);
    reduce_pairs_kernel<<<1, RED_THREADS, 0, st>>>(scratch, RED_CTAS, out);
}

int diff_norms_scratch_pairs() { return RED_CTAS; }

namespace {
int grid_for(size_t total) {
    size_t blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    return blocks < 1 ? 1 : (int)blocks;
}
}  // namespace

void complex_embed(int m, int n, const double* Z, int ldz, double* E, int lde, cudaStream_t st) {
    complex_embed_kernel<<<grid_for((size_t)m * n), 256, 0, st>>>(m, n, Z, ldz, E, lde);
}

void complex_extract(int r, int c, const double* E, int lde, double* Z, int ldz, cudaStream_t st) {
    complex_extract_kernel<<<grid_for((size_t)r * c), 256, 0, st>>>(r, c, E, lde, Z, ldz);
}

void embed_mirror(int M, int N2, double* E, int ld, cudaStream_t st) {
    embed_mirror_kernel<<<grid_for((size_t)(M / 2) * N2), 256, 0, st>>>(M, N2, E, ld);
}

void jacobi_x0(int n, const double* A, int lda, double alpha, double* X, int ldx, bool cplx, double* out,
               cudaStream_t st) {
    jacobi_x0_kernel<<<1, 256, 0, st>>>(n, A, lda, alpha, X, ldx, cplx ? 1 : 0, out);
}

void chop(int rows, int cols, double* X, int ld, double eps, cudaStream_t st) {
    chop_kernel<<<grid_for((size_t)rows * cols), 256, 0, st>>>(rows, cols, X, ld, eps);
}

void complex_norms_1_inf(int m, int n, const double* E, int lde, double* out, double* scratch, cudaStream_t st) {
    complex_col_abs_max_kernel<<<RED_CTAS, RED_THREADS, 0, st>>>(m, n, E, lde, scratch);
    max_kernel<<<1, RED_THREADS, 0, st>>>(scratch, RED_CTAS, out);
    complex_row_abs_max_kernel<<<RED_CTAS, RED_THREADS, 0, st>>>(m, n, E, lde, scratch + RED_CTAS);
    max_kernel<<<1, RED_THREADS, 0, st>>>(scratch + RED_CTAS, RED_CTAS, out + 1);
}

}  // namespace pinv
