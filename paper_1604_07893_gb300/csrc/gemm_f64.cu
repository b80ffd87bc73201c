// FP64 GEMM with the fused epilogue used by every product of the iteration.
//
// tcgen05 has no FP64 kind, so FP64 products run on the FP64 tensor path
// through mma.sync m8n8k4 (DMMA).  A CTA tile of 64x64, 32x32 or 16x16 with
// four warps in a 2x2 arrangement, BK = 16; the next K-slab is fetched into
// registers while the current one is multiplied from shared memory.  Ragged
// edges are zero-filled on load and masked on store, so any M, N, K >= 1 works.
// GB300's FP64 rate is about 2 FMA per clock per SM, so even a 16x16 tile is
// bound by the FP64 pipe, not by memory: small products take the smallest tile
// that still fills the GPU, which spreads them over the most SMs.
//
// The epilogue forms the linear combinations of Eq. PM directly from the
// accumulator (identity subtraction for R = I - AX, the I + c R2 + R4 factors,
// T, S, the TS + mu R2 + psi R4 sum, the update X + D X) and, optionally, the
// two Frobenius partial sums of the stop test (Eq. stopreliable / relative
// step).

#include "common.h"

namespace pinv {
namespace {

constexpr int BK = 16;
constexpr int APAD = 4;   // As row stride BK + APAD doubles: conflict-free fragment reads
constexpr int BPAD = 4;   // Bs row stride BN + BPAD
constexpr int THREADS = 128;

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

struct GemmArgs {
    int M, N, K;
    const double* A; int lda; int transA;
    const double* B; int ldb; int transB;
    long long stride;   // batch: instance b reads/writes every matrix at +b*stride
    int sym;            // symmetric output: only tiles with n-block >= m-block, mirrored
};

__device__ __forceinline__ double loadA(const GemmArgs& g, int i, int k) {
    if (i >= g.M || k >= g.K) return 0.0;
    return g.transA ? g.A[(size_t)k * g.lda + i] : g.A[(size_t)i * g.lda + k];
}
__device__ __forceinline__ double loadB(const GemmArgs& g, int k, int j) {
    if (k >= g.K || j >= g.N) return 0.0;
    return g.transB ? g.B[(size_t)j * g.ldb + k] : g.B[(size_t)k * g.ldb + j];
}

// BM x BN CTA tile (BM == BN); each of the four warps owns a (BM/2) x (BN/2)
// quadrant of (BM/16) x (BN/16) 8x8 accumulators.  BM = 8: one 8x8 tile per
// CTA whose four warps split each K-slab (one k-group of 4 each) and add
// their accumulators through shared memory at the end.
template <int BM, int BN>
__global__ void __launch_bounds__(THREADS)
gemm_f64_kernel(GemmArgs g, Epilogue epi) {
    constexpr bool KS = BM == 8;                        // K split across the warps
    constexpr int FM = KS ? 1 : BM / 16, FN = KS ? 1 : BN / 16;   // 8x8 fragments per warp
    constexpr int NA = BM * BK / THREADS, NB = BK * BN / THREADS;   // slab elements per thread
    __shared__ double As[BM][BK + APAD];
    __shared__ double Bs[BK][BN + BPAD];
    __shared__ double red[2][THREADS / 32];
    __shared__ double ksum[KS ? 4 : 1][32][2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = KS ? 0 : warp >> 1, wn = KS ? 0 : warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (g.sym && blockIdx.y > blockIdx.x) return;   // lower triangle: mirrored by its partner
    const bool mirror = g.sym && blockIdx.y != blockIdx.x;
    if (blockIdx.z) {   // instance blockIdx.z of a batch: shift every matrix
        const long long off = (long long)blockIdx.z * g.stride;
        g.A += off; g.B += off;
        if (epi.s1) epi.s1 += off;
        if (epi.s2) epi.s2 += off;
        for (int o = 0; o < 3; ++o)
            if (epi.o[o].out) epi.o[o].out += off;
        if (epi.partials) epi.partials += 2LL * blockIdx.z * gridDim.x * gridDim.y;
    }

    // Register staging of one K-slab: BM*BK A elements and BK*BN B elements.
    double ra[NA], rb[NB];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            int idx = tid + t * THREADS;
            int r, k;
            if (g.transA) { r = idx % BM; k = idx / BM; }   // consecutive threads: consecutive i
            else          { k = idx % BK; r = idx / BK; }   // consecutive threads: consecutive k
            ra[t] = loadA(g, m0 + r, k0 + k);
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            int idx = tid + t * THREADS;
            int kb, c;
            if (g.transB) { kb = idx % BK; c = idx / BK; }
            else          { c = idx % BN; kb = idx / BN; }
            rb[t] = loadB(g, k0 + kb, n0 + c);
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            int idx = tid + t * THREADS;
            int r, k;
            if (g.transA) { r = idx % BM; k = idx / BM; }
            else          { k = idx % BK; r = idx / BK; }
            As[r][k] = ra[t];
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            int idx = tid + t * THREADS;
            int kb, c;
            if (g.transB) { kb = idx % BK; c = idx / BK; }
            else          { c = idx % BN; kb = idx / BN; }
            Bs[kb][c] = rb[t];
        }
    };

    double acc[FM][FN][2];
#pragma unroll
    for (int i = 0; i < FM; ++i)
#pragma unroll
        for (int j = 0; j < FN; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    const int ktiles = (g.K + BK - 1) / BK;
    fetch(0);
    for (int kt = 0; kt < ktiles; ++kt) {
        __syncthreads();
        stash();
        __syncthreads();
        if (kt + 1 < ktiles) fetch((kt + 1) * BK);
#pragma unroll
        for (int kk = KS ? 4 * warp : 0; kk < BK; kk += KS ? BK : 4) {
            double af[FM], bf[FN];
#pragma unroll
            for (int i = 0; i < FM; ++i) af[i] = As[wm * (BM / 2) + i * 8 + (lane >> 2)][kk + (lane & 3)];
#pragma unroll
            for (int j = 0; j < FN; ++j) bf[j] = Bs[kk + (lane & 3)][wn * (BN / 2) + j * 8 + (lane >> 2)];
#pragma unroll
            for (int i = 0; i < FM; ++i)
#pragma unroll
                for (int j = 0; j < FN; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
        }
    }

    if constexpr (KS) {   // add the four warps' partial sums; warp 0 runs the epilogue
        ksum[warp][lane][0] = acc[0][0][0];
        ksum[warp][lane][1] = acc[0][0][1];
        __syncthreads();
        if (warp == 0)
            for (int w = 1; w < 4; ++w) { acc[0][0][0] += ksum[w][lane][0]; acc[0][0][1] += ksum[w][lane][1]; }
    }

    // ---- fused epilogue
    double sd = 0.0, sx = 0.0;
#pragma unroll
    for (int i = 0; i < FM && (!KS || warp == 0); ++i) {
        const int row = m0 + wm * (BM / 2) + i * 8 + (lane >> 2);
#pragma unroll
        for (int j = 0; j < FN; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = n0 + wn * (BN / 2) + j * 8 + 2 * (lane & 3) + h;
                if (row < g.M && col < g.N) {
                    const double a = acc[i][j][h];
                    const double v1 = epi.s1 ? epi.s1[(size_t)row * epi.ld1 + col] : 0.0;
                    const double v2 = epi.s2 ? epi.s2[(size_t)row * epi.ld2 + col] : 0.0;
                    const double id = (row == col) ? 1.0 : 0.0;
#pragma unroll
                    for (int o = 0; o < 3; ++o) {
                        if (o < epi.nout) {
                            const EpiTerm& t = epi.o[o];
                            double v = t.a_acc * a + t.a_s1 * v1 + t.a_s2 * v2 + t.a_id * id;
                            if (t.out) {
                                t.out[(size_t)row * t.ld + col] = v;
                                if (mirror) t.out[(size_t)col * t.ld + row] = v;
                            }
                            if (o == 0 && epi.partials) {
                                const double d = v - v1;
                                sd += d * d;
                                sx += v1 * v1;
                            }
                        }
                    }
                }
            }
        }
    }
    if (epi.partials) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            sd += __shfl_xor_sync(0xffffffffu, sd, off);
            sx += __shfl_xor_sync(0xffffffffu, sx, off);
        }
        if (lane == 0) { red[0][warp] = sd; red[1][warp] = sx; }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < THREADS / 32; ++w) { a += red[0][w]; b += red[1][w]; }
            const int cta = blockIdx.y * gridDim.x + blockIdx.x;
            epi.partials[2 * cta] = a;
            epi.partials[2 * cta + 1] = b;
        }
    }
}

}  // namespace

int gemm_f64_ctas(int M, int N, int tile) { return ((N + tile - 1) / tile) * ((M + tile - 1) / tile); }

int gemm_f64_pick_tile(int M, int N, int batch, int sms) {
    for (int tile : {64, 32, 16})
        if ((long long)gemm_f64_ctas(M, N, tile) * batch >= sms) return tile;
    return 8;
}

int gemm_f64(int M, int N, int K, const double* A, int lda, bool transA,
             const double* B, int ldb, bool transB, const Epilogue& epi, cudaStream_t st,
             int batch, long long stride, bool sym_out, int tile) {
    if (sym_out && (M != N || epi.partials)) return -1;
    GemmArgs g{M, N, K, A, lda, transA ? 1 : 0, B, ldb, transB ? 1 : 0, stride, sym_out ? 1 : 0};
    dim3 grid((N + tile - 1) / tile, (M + tile - 1) / tile, batch);
    if (tile == 64) gemm_f64_kernel<64, 64><<<grid, THREADS, 0, st>>>(g, epi);
    else if (tile == 32) gemm_f64_kernel<32, 32><<<grid, THREADS, 0, st>>>(g, epi);
    else if (tile == 16) gemm_f64_kernel<16, 16><<<grid, THREADS, 0, st>>>(g, epi);
    else if (tile == 8) gemm_f64_kernel<8, 8><<<grid, THREADS, 0, st>>>(g, epi);
    else return -1;
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    return grid.x * grid.y;   // pair partials per instance
}

}  // namespace pinv
