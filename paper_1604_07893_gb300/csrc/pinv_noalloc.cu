// pinv_step_noalloc: one FP64 loop of the iteration without any allocation.
//
// Who needs it: code that runs where device allocation is not available or
// not allowed -- a plugin handed buffers by a host framework that owns the
// allocator, code running under a memory pool that forbids cudaMalloc, or a
// process that must not trigger the implicit device synchronisation that
// cudaMalloc/cudaFree can cause.  Such a caller passes A, X_in and X_out and
// this entry point takes every intermediate (R, R2, R4, the L1/L2/T/S/Z/D
// squares, the half step of the stabilised loop, the stop-norm partials) from
// one static device array of fixed size, so it never calls cudaMalloc,
// cudaFree, cudaMallocHost or any allocating library routine.
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds it until the process exits.  Host code cannot use its name as
// a device address (the name denotes a host-side shadow), so the device
// address is looked up once per device with cudaGetSymbolAddress on the first
// call made on that device.
//
// Limits and sharing rules:
//   * m and n must both be <= PINV_NOALLOC_MAX_DIM (128); larger shapes are
//     rejected with PINV_ERR_BUDGET before any device work.
//   * All calls on a device share the one array.  Calls that overlap on the
//     GPU (different streams, or host threads) race on it: serialise them.
//   * The array keeps the previous call's contents; every scratch word this
//     call reads is first written by this call, and the stop-norm slots are
//     cleared at the start of each call.

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/pinv.h"
#include "common.h"

using namespace pinv;

namespace {

constexpr int kMaxDim = PINV_NOALLOC_MAX_DIM;
constexpr size_t kSquare = (size_t)kMaxDim * kMaxDim;      // doubles in one square
// Every product runs on the DMMA kernel with this CTA tile, one stop-norm pair
// per CTA; the partial slots below are sized for it (and checked per call).
constexpr int kTile = 64;
constexpr int kMaxTiles = ((kMaxDim + kTile - 1) / kTile) * ((kMaxDim + kTile - 1) / kTile);
// 7 squares (R, R2, R4, L1, L2, T, S), one n x m half step, 2 partials per CTA,
// two reduced norms.
constexpr size_t kScratchDoubles = 8 * kSquare + 2 * kMaxTiles + 2;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PINV_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            std::fprintf(stderr, "pinv_step_noalloc: cudaGetSymbolAddress failed: %s\n",
                         cudaGetErrorString(e));
            return PINV_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return PINV_OK;
}

EpiTerm term(double* out, int ld, double a_acc, double a_s1 = 0, double a_s2 = 0, double a_id = 0) {
    EpiTerm t;
    t.out = out; t.ld = ld; t.a_acc = a_acc; t.a_s1 = a_s1; t.a_s2 = a_s2; t.a_id = a_id;
    return t;
}
Epilogue epi(EpiTerm t0, const double* s1 = nullptr, int ld1 = 0, const double* s2 = nullptr,
             int ld2 = 0) {
    Epilogue e{};
    e.s1 = s1; e.ld1 = ld1; e.s2 = s2; e.ld2 = ld2;
    e.o[0] = t0; e.nout = 1; e.partials = nullptr;
    return e;
}

}  // namespace

extern "C" int pinv_step_noalloc(int m, int n, const double* A, int lda, const double* X_in,
                                 double* X_out, int ldx, int stabilized, void* stream,
                                 double* rel_step) {
    if (m < 1 || n < 1 || !A || !X_in || !X_out || lda < n || ldx != m || X_in == X_out)
        return PINV_ERR_ARG;
    if (m > kMaxDim || n > kMaxDim) {
        std::fprintf(stderr, "pinv_step_noalloc: %d x %d exceeds the static scratch limit of %d x %d\n",
                     m, n, kMaxDim, kMaxDim);
        return PINV_ERR_BUDGET;
    }
    // the stop-norm partials come from the n x m update product: one pair per CTA
    if (gemm_f64_ctas(n, m, kTile) > kMaxTiles) return PINV_ERR_BUDGET;
    double* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    const bool left = m > n;
    const int s = left ? n : m;
    double* sq[7];
    for (int i = 0; i < 7; ++i) sq[i] = base + i * kSquare;
    double* Xh = base + 7 * kSquare;
    double* partials = base + 8 * kSquare;
    double* norms = partials + 2 * kMaxTiles;
    if (cudaMemsetAsync(partials, 0, sizeof(double) * (2 * kMaxTiles + 2), st) != cudaSuccess)
        return PINV_ERR_CUDA;

    // Section 2 closed forms
    const double r93 = std::sqrt(93.0), q = std::sqrt(27.0 - 2.0 * r93);
    const double c1 = 0.25 * (1.0 + q), c2 = 0.25 * (1.0 - q), c3 = (5.0 * r93 - 93.0) / 496.0;
    const double d1 = (-93.0 - 5.0 * r93) / 496.0, d2 = -0.25 * r93, mu = 3.0 / 8.0,
                 psi = 321.0 / 1984.0;
    double *R = sq[0], *R2 = sq[1], *R4 = sq[2], *L1 = sq[3], *L2 = sq[4], *T = sq[5], *S = sq[6];
    double *Z = L1, *D = L2;
    double* target = stabilized ? Xh : X_out;

    bool ok = true;
    auto G = [&](int M, int N, int K, const double* a, int la, bool ta, const double* b, int lb,
                 bool tb, const Epilogue& e) {
        int r = gemm_f64(M, N, K, a, la, ta, b, lb, tb, e, st, 1, 0, false, kTile);
        if (r < 0) ok = false;
        return r;
    };
    // Eq. PM: the seven products with fused combinations
    if (left) G(s, s, m, X_in, m, false, A, lda, false, epi(term(R, s, -1, 0, 0, 1)));
    else      G(s, s, n, A, lda, false, X_in, m, false, epi(term(R, s, -1, 0, 0, 1)));
    G(s, s, s, R, s, false, R, s, false, epi(term(R2, s, 1)));
    {
        Epilogue e = epi(term(R4, s, 1), R2, s);
        e.o[1] = term(L1, s, 1, c1, 0, 1);
        e.o[2] = term(L2, s, 1, c2, 0, 1);
        e.nout = 3;
        G(s, s, s, R2, s, false, R2, s, false, e);
    }
    {
        Epilogue e = epi(term(T, s, 1, c3), R2, s, R4, s);
        e.o[1] = term(S, s, 1, d1, d2);
        e.nout = 2;
        G(s, s, s, L1, s, false, L2, s, false, e);
    }
    G(s, s, s, T, s, false, S, s, false, epi(term(Z, s, 1, mu, psi), R2, s, R4, s));
    G(s, s, s, R, s, false, Z, s, false, epi(term(D, s, 1, 1, 0, -1), Z, s));
    Epilogue up = epi(term(target, m, 1, 1), X_in, m);
    up.partials = stabilized ? nullptr : partials;
    int parts = left ? G(n, m, s, D, s, false, X_in, m, false, up)
                     : G(n, m, s, X_in, m, false, D, s, false, up);
    if (stabilized) {  // Eq. PM-modified: X_out = Xh A Xh, smaller square in the middle
        double* P = T;
        Epilogue fin = epi(term(X_out, m, 1), X_in, m);
        fin.partials = partials;
        if (left) {
            G(s, s, m, Xh, m, false, A, lda, false, epi(term(P, s, 1)));
            parts = G(n, m, s, P, s, false, Xh, m, false, fin);
        } else {
            G(s, s, n, A, lda, false, Xh, m, false, epi(term(P, s, 1)));
            parts = G(n, m, s, Xh, m, false, P, s, false, fin);
        }
    }
    if (!ok || parts < 0) return PINV_ERR_CUDA;
    reduce_pairs(partials, parts, norms, st);
    // a failed launch of this call is reported here; errors left behind by
    // other code are neither reported nor cleared
    if (cudaPeekAtLastError() != cudaSuccess) return PINV_ERR_CUDA;
    double h[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PINV_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PINV_ERR_CUDA;
    if (rel_step) *rel_step = h[1] > 0 ? std::sqrt(h[0] / h[1]) : INFINITY;
    return PINV_OK;
}
