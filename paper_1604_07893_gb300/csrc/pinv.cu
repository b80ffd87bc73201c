// Host driver of the C ABI declared in include/pinv.h.
//
// One solve = X0 (Section 4) followed by loops of the factorised step of
// Eq. PM, each a fixed chain of seven fused-epilogue GEMM launches on the
// caller's stream:
//   1  R  = I - X A         (left, n x n)      or  I - A X   (right, m x m)
//   2  R2 = R R
//   3  R4 = R2 R2,   L1 = I + c1 R2 + R4,   L2 = I + c2 R2 + R4
//   4  M  = L1 L2 ->  T = M + c3 R2,   S = M + d1 R2 + d2 R4
//   5  Z  = T S + mu R2 + psi R4
//   6  D  = R Z + Z - I                    ((I + R) Z = I + D)
//   7  X' = X + D X         (left)          or  X + X D     (right)
//      + Frobenius partials of X' - X and X for the stop test.
// The stabilised loop (Eq. PM-modified) adds X' <- X' A X' as two more GEMMs,
// ordered so the middle product is the smaller square.  Only the two stop
// norms come back to the host per loop.

#include <algorithm>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/pinv.h"
#include "common.h"
#include "tc_gemm.h"

using namespace pinv;

namespace {

// Closed forms of Section 2 for the parameters of Eq. simplify1/simplify2 and
// Eq. hyper18-33 (c1, c2, c3, d1, d2, mu, psi).
struct Coef {
    double c1, c2, c3, d1, d2, mu, psi;
};
Coef pm_coefficients() {
    const double r93 = std::sqrt(93.0);
    const double q = std::sqrt(27.0 - 2.0 * r93);
    Coef c;
    c.c1 = 0.25 * (1.0 + q);
    c.c2 = 0.25 * (1.0 - q);
    c.c3 = (5.0 * r93 - 93.0) / 496.0;
    c.d1 = (-93.0 - 5.0 * r93) / 496.0;
    c.d2 = -0.25 * r93;
    c.mu = 3.0 / 8.0;
    c.psi = 321.0 / 1984.0;
    return c;
}

EpiTerm term(double* out, int ld, double a_acc, double a_s1 = 0, double a_s2 = 0, double a_id = 0) {
    EpiTerm t;
    t.out = out; t.ld = ld; t.a_acc = a_acc; t.a_s1 = a_s1; t.a_s2 = a_s2; t.a_id = a_id;
    return t;
}
Epilogue epi1(EpiTerm t0, const double* s1 = nullptr, int ld1 = 0, const double* s2 = nullptr,
              int ld2 = 0) {
    Epilogue e{};
    e.s1 = s1; e.ld1 = ld1; e.s2 = s2; e.ld2 = ld2;
    e.o[0] = t0; e.nout = 1; e.partials = nullptr;
    return e;
}

}  // namespace

// State of a solve whose loop runs on the device (a graph WHILE node): the
// stop rule's inputs and outputs, written by the host before the launch and
// read back after it.
struct DeviceLoopState {
    int k, max_iter, stop_mode, status, reason, iters, loops_run, copy;
    double alpha, tol, prev, prev2, rel_step;
    double history[PINV_HISTORY];
};

struct pinv_handle {
    int device = 0;
    size_t budget = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    double* pinned = nullptr;  // host pinned readback block
    double* dsmall = nullptr;  // device: reduction outputs
    int* derr = nullptr;       // device error word of the tensor-core kernels
    unsigned wait_limit = 0;   // polls of a tensor-core kernel wait (0: the default)
    int tc_crossover = 0;      // pinv_autotune: FP64-class products below this size use DMMA
    int sms = 1;               // streaming multiprocessors of the device
    std::vector<cudaEvent_t> events;  // profiling pool (pairs), created on demand
    // small single solves replay their loop as a captured CUDA graph; the graph
    // refers to workspace buffers only, so it is reused by every later solve
    // whose loop touches the same buffers (key: those pointers, shapes, flags)
    struct LoopGraph {
        std::vector<long long> key;
        cudaGraphExec_t exec = nullptr;
        int kernels = 0, gemms = 0;
    };
    std::vector<LoopGraph> loop_graphs;
    cudaStream_t capture_stream = nullptr;    // graphs are captured here, replayed on the caller's stream
    DeviceLoopState* dstate = nullptr;        // device-driven loops: state on the device
    DeviceLoopState* hstate = nullptr;        // and its pinned host copy
    bool device_loop_off = false;             // set if such a graph could not be built here
    // pinned readback blocks for groups, reused (pinned allocation can
    // synchronise the device, so it happens only when the pool is empty)
    std::vector<void*> pinned_blocks;
    bool pool_ready = false;
    // serving (pinv_submit / pinv_poll)
    std::mutex mu;
    uint64_t next_id = 1;
    struct Request {
        pinv_desc desc;
        int status = PINV_PENDING;
        pinv_info info{};
        std::chrono::steady_clock::time_point t_submit;
    };
    std::deque<uint64_t> queue;                 // submitted, not yet admitted
    int max_queued = 0;                         // admission-queue cap (0: none)
    uint64_t n_submitted = 0, n_rejected = 0, n_admitted = 0, n_completed = 0;
    int n_running = 0;                          // admitted requests not yet completed
    std::map<uint64_t, Request> requests;
    struct Running;                             // a group of admitted requests on the device
    std::vector<std::unique_ptr<Running>> running;
    size_t serving_bytes = 0;                   // device memory held by running groups
};

namespace {

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            std::fprintf(stderr, "pinv: %s failed: %s (%s:%d)\n", #call,               \
                         cudaGetErrorString(e_), __FILE__, __LINE__);                  \
            return PINV_ERR_CUDA;                                                      \
        }                                                                              \
    } while (0)

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Everything one solve needs on the device.
struct Ctx {
    pinv_handle* h;
    cudaStream_t st;
    int m, n;         // A is m x n
    int s;            // residual dimension
    bool left;        // left residual I - XA
    const double* A; int lda;
    double* X[3];     // ping, pong, half-step; each n x m, ld = m
    double* sq[7];    // R R2 R4 L1 L2 T S; s x s, ld = s
    double* Al;       // A^l (Drazin), n x n
    double* Ad;       // device copy of A (host_buffers)
    double* Gd;       // device copy of G (host_buffers)
    double* big[2];   // max(m,n)^2 scratch for residual checks
    double* partials; // pair partials
    double* red;      // reduction scratch (2 * 256 pairs)
    int prec_k = 0;         // product precision of the GEMMs being issued (0 = DMMA FP64)
    int batch = 1;          // instances processed together (all buffers at +b*stride)
    long long stride = 0;
    bool yield_sms = false; // tensor-core launches release SMs after every tile
    bool symmetric = false; // R and its polynomials are symmetric: half the tiles, mirrored
    void* tcws = nullptr;   // slice workspace of the tensor-core engine
    size_t tcws_bytes = 0;
    int gemms = 0;
    bool replay = false;    // loops replayed from cached graphs (A copied into the workspace)
    bool cplx = false;      // complex problem solved as its real embedding (m, n above are 2x)
    int kernels = 0;
    bool profile = false;
    int ev_used = 0;        // event pairs recorded since the last harvest
    double gemm_flops = 0;
    double tensor_flops = 0;
    float gemm_ms = 0;
    Coef c;
};

// Time GEMM kernels with CUDA events on the launch stream; harvested at sync
// points.  For the tensor-core engine the events bracket the tcgen05 kernel
// alone (not the slicing kernels before it).
int prof_slot(Ctx& c) {
    if (!c.profile) return -1;
    auto& ev = c.h->events;
    if ((int)ev.size() < 2 * (c.ev_used + 1)) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            ev.push_back(e);
        }
    }
    return c.ev_used++;
}
cudaEvent_t prof_ev(Ctx& c, int slot, int which) {
    return slot >= 0 ? c.h->events[2 * slot + which] : nullptr;
}
void prof_harvest(Ctx& c) {  // stream already synchronised
    for (int i = 0; i < c.ev_used; ++i) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c.h->events[2 * i], c.h->events[2 * i + 1]) == cudaSuccess)
            c.gemm_ms += ms;
    }
    c.ev_used = 0;
}

size_t tc_bytes(int m, int n, int prec) {
    const int big = std::max(m, n);
    return prec == PINV_PREC_FP64 ? 0 : tc_workspace_bytes(big, big, big, tc_mode(TC_FP64));
}

size_t workspace_bytes(int m, int n, bool drazin, bool host, bool check, int prec) {
    // `check` also covers the finish step: both need the two max(m,n)^2 squares
    const size_t s = std::min(m, n), big = std::max(m, n);
    size_t b = 0;
    b += 3 * align_up(sizeof(double) * n * (size_t)m);
    b += 7 * align_up(sizeof(double) * s * s);
    if (drazin) b += align_up(sizeof(double) * n * (size_t)n);
    if (host) b += 2 * align_up(sizeof(double) * n * (size_t)m);
    if (check) b += 2 * align_up(sizeof(double) * big * big);
    b += align_up(sizeof(double) * 2 * partial_pairs_bound(big, big));   // stop-norm pair partials
    b += align_up(sizeof(double) * 2 * 2 * 256);
    b += align_up(tc_bytes(m, n, prec));
    return b;
}

int ensure_workspace(pinv_handle* h, size_t bytes) {
    if (h->budget && bytes > h->budget) return PINV_ERR_BUDGET;
    if (bytes <= h->ws_bytes) return PINV_OK;
    for (auto& g : h->loop_graphs) cudaGraphExecDestroy(g.exec);   // they refer to the old workspace
    h->loop_graphs.clear();
    if (h->ws) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(h->ws));
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    CK(cudaMalloc(&h->ws, bytes));
    h->ws_bytes = bytes;
    return PINV_OK;
}

void carve(Ctx& c, bool drazin, bool host, bool check, int prec) {
    char* p = c.h->ws;
    auto take = [&](size_t bytes) { char* q = p; p += align_up(bytes); return (double*)q; };
    const size_t s = c.s, big = std::max(c.m, c.n);
    for (int i = 0; i < 3; ++i) c.X[i] = take(sizeof(double) * c.n * (size_t)c.m);
    for (int i = 0; i < 7; ++i) c.sq[i] = take(sizeof(double) * s * s);
    c.Al = drazin ? take(sizeof(double) * c.n * (size_t)c.n) : nullptr;
    c.Ad = host ? take(sizeof(double) * c.n * (size_t)c.m) : nullptr;
    c.Gd = host ? take(sizeof(double) * c.n * (size_t)c.m) : nullptr;
    c.big[0] = check ? take(sizeof(double) * big * big) : nullptr;
    c.big[1] = check ? take(sizeof(double) * big * big) : nullptr;
    c.partials = take(sizeof(double) * 2 * partial_pairs_bound(big, big));
    c.red = take(sizeof(double) * 2 * 2 * 256);
    c.tcws_bytes = tc_bytes(c.m, c.n, prec);
    c.tcws = c.tcws_bytes ? (void*)take(c.tcws_bytes) : nullptr;
}

int gemm(Ctx& c, int M, int N, int K, const double* A, int lda, bool tA, const double* B, int ldb,
         bool tB, const Epilogue& e, bool sym = false) {
    // Complex problems: every matrix is held as its embedding E(Z) =
    // [[Re Z, -Im Z], [Im Z, Re Z]], and E(C) = E(A) E(B).  The left column half
    // of E(C), [Re C; Im C], needs only the left half of E(B) (the 4M complex
    // product: half the work of the full real product); a mirror kernel writes
    // the right half.  The epilogue sees the left half only, so its stop-norm
    // partials are the complex Frobenius norms.
    if (c.cplx) {
        N /= 2;
        sym = false;
    }
    ++c.gemms;
    ++c.kernels;
    c.gemm_flops += 2.0 * M * N * K * c.batch;   // algorithmic work of the full product
    const int slot = prof_slot(c);
    int r;
    // autotuned engine choice: small FP64-class products run on the DMMA kernel
    const bool small = c.prec_k == TC_FP64 && std::max(M, std::max(N, K)) < c.h->tc_crossover;
    if (c.prec_k == 0 || small) {
        if (slot >= 0) cudaEventRecord(prof_ev(c, slot, 0), c.st);
        r = gemm_f64(M, N, K, A, lda, tA, B, ldb, tB, e, c.st, c.batch, c.stride, sym,
                     gemm_f64_pick_tile(M, N, c.batch, c.h->sms));
        if (slot >= 0) cudaEventRecord(prof_ev(c, slot, 1), c.st);
    } else {
        --c.kernels;  // tc_gemm counts its own launches (slicing + GEMM)
        {
            const int tm = (M + 127) / 128;   // executed tiles: the upper triangle in symmetric mode
            const double frac = sym ? (double)(tm * (tm + 1) / 2) / (double)(tm * tm) : 1.0;
            c.tensor_flops += 2.0 * M * N * K * tc_pairs(tc_mode(c.prec_k)) * c.batch * frac;
        }
        r = tc_gemm(M, N, K, A, lda, tA, B, ldb, tB, e, tc_mode(c.prec_k), c.tcws, c.tcws_bytes,
                    c.h->derr, c.st, &c.kernels, prof_ev(c, slot, 0), prof_ev(c, slot, 1), c.batch,
                    c.stride, c.yield_sms, sym, c.h->wait_limit);
    }
    if (c.cplx && r >= 0) {
        for (int o = 0; o < e.nout; ++o) {
            if (!e.o[o].out) continue;
            embed_mirror(M, N, e.o[o].out, e.o[o].ld, c.st);
            ++c.kernels;
        }
    }
    return r;
}

// Read the two stop norms (sum of squares) reduced from `count` pair partials.
int read_norms(Ctx& c, int count, double* dx2, double* x2) {
    reduce_pairs(c.partials, count, c.h->dsmall, c.st);
    ++c.kernels;
    CK(cudaMemcpyAsync(c.h->pinned, c.h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    CK(cudaMemcpyAsync(c.h->pinned + 2, c.h->derr, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    prof_harvest(c);
    *dx2 = c.h->pinned[0];
    *x2 = c.h->pinned[1];
    int derr;
    std::memcpy(&derr, c.h->pinned + 2, sizeof(int));
    if (derr) {
        std::fprintf(stderr, "pinv: tensor-core kernel wait timed out (code %d)\n", derr);
        cudaMemsetAsync(c.h->derr, 0, sizeof(int), c.st);
        return PINV_ERR_TIMEOUT;
    }
    return PINV_OK;
}

// Precision schedule (monotone): the product class of the next loop from the
// class of the last loop and its relative step `rel` (||X_{k+1}-X_k||/||X_k||).
//  * BF16 serves the growth phase while the step is above 0.5 (problems
//    without a null block only: on a rank-deficient problem BF16 rounding lands
//    in the null block, which grows by 18 per loop, Theorem 6.2).
//  * FP32-class loops run while the iterate still grows (step >= 1); after the
//    first FP32-class loop whose step is below 1 the iterate is within one
//    order-18 contraction of its limit, and every later loop runs in the final
//    class: that loop takes the remaining error e to e^18 and removes the
//    FP32-class rounding of the range block at the same time.  Requires
//    alpha <= 1/sigma_max^2 (with 2/(sigma_1^2 + sigma_r^2) the top residual
//    eigenvalue sits at -1 and FP32-class rounding pushes it past).
int next_level(int level, int last_level, int final_class, double rel) {
    if (level == TC_BF16) return rel <= 0.5 ? TC_FP32 : level;
    if (level == TC_FP32 && final_class != TC_FP32 && last_level == TC_FP32 && rel < 1.0) return final_class;
    return level;
}

// One order-2 step of the hyperpower family (p = 2): X' = X + R X (left) or
// X + X R, R = I - XA | I - AX; it squares the residual with two products.
// The finish uses it after the projection unless BF16 loops ran: the
// projection's error is then first-order rounding (of FP64- or FP32-class
// loops), which one squaring removes.  After BF16 loops the projection leaves
// the second-order remainder of their persistent off-diagonal blocks (up to
// ~1e-2), and a full order-18 loop follows instead.

int ns_step_f64(Ctx& c, const double* Xin, double* Xout) {
    const int s = c.s, m = c.m, n = c.n;
    double* R = c.sq[0];
    if (c.left) gemm(c, s, s, m, Xin, m, false, c.A, c.lda, false, epi1(term(R, s, -1, 0, 0, 1)));
    else        gemm(c, s, s, n, c.A, c.lda, false, Xin, m, false, epi1(term(R, s, -1, 0, 0, 1)));
    Epilogue e = epi1(term(Xout, m, 1, 1), Xin, m);
    e.partials = c.partials;
    if (c.left) return gemm(c, n, m, s, R, s, false, Xin, m, false, e);
    return gemm(c, n, m, s, Xin, m, false, R, s, false, e);
}

int pm_loop_f64(Ctx& c, const double* Xin, double* Xout) {
    const int s = c.s, m = c.m, n = c.n;
    double *R = c.sq[0], *R2 = c.sq[1], *R4 = c.sq[2], *L1 = c.sq[3], *L2 = c.sq[4], *T = c.sq[5],
           *S = c.sq[6];
    double *Z = L1, *D = L2;  // L1/L2 are dead once M is formed
    const Coef& k = c.c;
    // With a symmetric A and a commuting G the exact R is symmetric.  R itself
    // and R Z are computed in full: their antisymmetric part is the first-order
    // correction of the iterate's error (near convergence R = -E11 Sigma), and
    // dropping it stops the self-correction (measured: 1e-6 errors after the
    // finish).  Products 2-5 only build the even polynomial of R, where
    // symmetrising drops second-order terms: they compute half their tiles.
    const bool y = c.symmetric;
    // 1: R = I - X A  |  I - A X
    if (c.left) gemm(c, s, s, m, Xin, m, false, c.A, c.lda, false, epi1(term(R, s, -1, 0, 0, 1)));
    else        gemm(c, s, s, n, c.A, c.lda, false, Xin, m, false, epi1(term(R, s, -1, 0, 0, 1)));
    // 2: R2
    gemm(c, s, s, s, R, s, false, R, s, false, epi1(term(R2, s, 1)), y);
    // 3: R4, L1, L2
    {
        Epilogue e = epi1(term(R4, s, 1), R2, s);
        e.o[1] = term(L1, s, 1, k.c1, 0, 1);
        e.o[2] = term(L2, s, 1, k.c2, 0, 1);
        e.nout = 3;
        gemm(c, s, s, s, R2, s, false, R2, s, false, e, y);
    }
    // 4: M = L1 L2 -> T, S
    {
        Epilogue e = epi1(term(T, s, 1, k.c3), R2, s, R4, s);
        e.o[1] = term(S, s, 1, k.d1, k.d2);
        e.nout = 2;
        gemm(c, s, s, s, L1, s, false, L2, s, false, e, y);
    }
    // 5: Z = T S + mu R2 + psi R4
    gemm(c, s, s, s, T, s, false, S, s, false, epi1(term(Z, s, 1, k.mu, k.psi), R2, s, R4, s), y);
    // 6: D = R Z + Z - I
    gemm(c, s, s, s, R, s, false, Z, s, false, epi1(term(D, s, 1, 1, 0, -1), Z, s));
    // 7: X' = X + D X | X + X D, with stop partials
    Epilogue e = epi1(term(Xout, m, 1, 1), Xin, m);
    e.partials = c.partials;
    int ctas;
    if (c.left) ctas = gemm(c, n, m, s, D, s, false, Xin, m, false, e);
    else        ctas = gemm(c, n, m, s, Xin, m, false, D, s, false, e);
    return ctas;
}

// X A X with the smaller square in the middle; partials against Xprev.
int stabilise_f64(Ctx& c, const double* Xh, const double* Xprev, double* Xout) {
    const int s = c.s, m = c.m, n = c.n;
    double* P = c.sq[5];
    Epilogue e = epi1(term(Xout, m, 1), Xprev, m);
    e.partials = c.partials;
    if (c.left) {  // P = Xh A (n x n); X' = P Xh
        gemm(c, s, s, m, Xh, m, false, c.A, c.lda, false, epi1(term(P, s, 1)));
        return gemm(c, n, m, s, P, s, false, Xh, m, false, e);
    }
    // Q = A Xh (m x m); X' = Xh Q
    gemm(c, s, s, n, c.A, c.lda, false, Xh, m, false, epi1(term(P, s, 1)));
    return gemm(c, n, m, s, Xh, m, false, P, s, false, e);
}

// Projection of the finish step: (XA)^T X (AX)^T (Moore-Penrose),
// A^l X^{2l+1} A^l (Drazin) or X A X (general G).  Xin -> Xout.
void cleanup_f64(Ctx& c, const pinv_desc* d, const double* X, double* Xout) {
    const int s = c.s, m = c.m, n = c.n;
    if (d->kind == PINV_DRAZIN || d->kind == PINV_DRAZIN_NORMAL) {
        const int l = d->drazin_index;
        double* V[2] = {c.sq[0], c.sq[1]};
        scale_copy(n, n, X, m, 1.0, V[0], n, c.st);
        ++c.kernels;
        int cur = 0;
        for (int i = 0; i < 2 * l; ++i) {
            gemm(c, n, n, n, V[cur], n, false, X, m, false, epi1(term(V[cur ^ 1], n, 1)));
            cur ^= 1;
        }
        gemm(c, n, n, n, c.Al, n, false, V[cur], n, false, epi1(term(V[cur ^ 1], n, 1)));
        gemm(c, n, n, n, V[cur ^ 1], n, false, c.Al, n, false, epi1(term(Xout, m, 1)));
        return;
    }
    if (d->kind == PINV_OUTER_G) {
        // X' = X A X: XAX = X defines every outer inverse (Eq. 1), so it fixes
        // A^(2)_{T,S} for any G and removes the error components outside R(X)
        // (left) and N(X) (right); the Moore-Penrose projection below would move
        // a non-Moore-Penrose outer inverse (e.g. a weighted one) off itself.
        double* P = c.sq[5];
        if (c.left) {   // P = XA (n x n), X' = P X
            gemm(c, n, n, m, X, m, false, c.A, c.lda, false, epi1(term(P, n, 1)));
            gemm(c, n, m, n, P, n, false, X, m, false, epi1(term(Xout, m, 1)));
        } else {        // Q = AX (m x m), X' = X Q
            gemm(c, m, m, n, c.A, c.lda, false, X, m, false, epi1(term(P, m, 1)));
            gemm(c, n, m, m, X, m, false, P, m, false, epi1(term(Xout, m, 1)));
        }
        return;
    }
    // X' = P^T X Q^T with P = XA (n x n) and Q = AX (m x m): both factors are
    // near-projectors (entries O(1)), so no intermediate grows like ||X||^2.
    double *P = c.big[0], *Q = c.big[1], *Y = c.X[2];
    gemm(c, n, n, m, X, m, false, c.A, c.lda, false, epi1(term(P, n, 1)));
    gemm(c, m, m, n, c.A, c.lda, false, X, m, false, epi1(term(Q, m, 1)));
    gemm(c, n, m, n, P, n, true, X, m, false, epi1(term(Y, m, 1)));
    gemm(c, n, m, m, Y, m, false, Q, m, true, epi1(term(Xout, m, 1)));
    (void)s;
}

// Relative residual norms of the Penrose (Moore-Penrose / general) or Drazin
// equations for the final X.
int residual_checks(Ctx& c, const pinv_desc* d, const double* X, pinv_info* info) {
    const int m = c.m, n = c.n;
    double* AX = c.big[0];   // m x m
    double* XA = c.big[1];   // n x n
    double v[2];
    auto norms = [&](int count) -> int {
        double a, b;
        int rc = read_norms(c, count, &a, &b);
        v[0] = a; v[1] = b;
        return rc;
    };
    gemm(c, m, m, n, c.A, c.lda, false, X, m, false, epi1(term(AX, m, 1)));
    gemm(c, n, n, m, X, m, false, c.A, c.lda, false, epi1(term(XA, n, 1)));
    if (d->kind == PINV_DRAZIN || d->kind == PINV_DRAZIN_NORMAL) {
        const int l = d->drazin_index;
        // ||XAX - X|| / ||X||
        Epilogue e = epi1(term(nullptr, 0, 1), X, m);
        e.partials = c.partials;
        int k = gemm(c, n, m, n, XA, n, false, X, m, false, e);
        if (norms(k)) return PINV_ERR_CUDA;
        info->drazin[0] = std::sqrt(v[0] / v[1]);
        // ||AX - XA|| / ||AX||
        diff_norms(n, n, AX, m, XA, n, false, c.h->dsmall, c.red, c.st);
        c.kernels += 2;
        CK(cudaMemcpyAsync(c.h->pinned, c.h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
        CK(cudaStreamSynchronize(c.st));
        info->drazin[1] = std::sqrt(c.h->pinned[0] / c.h->pinned[1]);
        // ||A^l (AX) - A^l|| / ||A^l||
        e = epi1(term(nullptr, 0, 1), c.Al, n);
        e.partials = c.partials;
        k = gemm(c, n, n, n, c.Al, n, false, AX, m, false, e);
        if (norms(k)) return PINV_ERR_CUDA;
        info->drazin[2] = std::sqrt(v[0] / v[1]);
        (void)l;
        return PINV_OK;
    }
    // ||AXA - A|| / ||A||
    Epilogue e = epi1(term(nullptr, 0, 1), c.A, c.lda);
    e.partials = c.partials;
    int k = gemm(c, m, n, m, AX, m, false, c.A, c.lda, false, e);
    if (norms(k)) return PINV_ERR_CUDA;
    info->penrose[0] = std::sqrt(v[0] / v[1]);
    // ||X AX - X|| / ||X||
    e = epi1(term(nullptr, 0, 1), X, m);
    e.partials = c.partials;
    k = gemm(c, n, m, m, X, m, false, AX, m, false, e);
    if (norms(k)) return PINV_ERR_CUDA;
    info->penrose[1] = std::sqrt(v[0] / v[1]);
    // ||AX - (AX)^T|| / ||AX||, ||XA - (XA)^T|| / ||XA||
    diff_norms(m, m, AX, m, AX, m, true, c.h->dsmall, c.red, c.st);
    c.kernels += 2;
    CK(cudaMemcpyAsync(c.h->pinned, c.h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    info->penrose[2] = std::sqrt(c.h->pinned[0] / c.h->pinned[1]);
    diff_norms(n, n, XA, n, XA, n, true, c.h->dsmall, c.red, c.st);
    c.kernels += 2;
    CK(cudaMemcpyAsync(c.h->pinned, c.h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    info->penrose[3] = std::sqrt(c.h->pinned[0] / c.h->pinned[1]);
    return PINV_OK;
}

// The caller's hint: a symmetric A with a G that commutes with it (e.g. G = I),
// so the exact iterates are polynomials in A and R is symmetric.  Not used for
// Moore-Penrose: on rank-deficient problems even the symmetrised even
// polynomial loses accuracy (6e-9 instead of 2e-12 on 512 x 384 rank 288).
bool iterates_symmetric(const pinv_desc* d) {
    return d->kind == PINV_OUTER_G && d->symmetric;
}

int validate(const pinv_desc* d) {
    if (!d) return PINV_ERR_ARG;
    if (d->m < 1 || d->n < 1) return PINV_ERR_ARG;
    if (!d->A || !d->X) return PINV_ERR_ARG;
    if (d->lda < d->n || d->ldx < d->m) return PINV_ERR_ARG;
    if ((d->kind == PINV_DRAZIN || d->kind == PINV_DRAZIN_NORMAL) && (d->m != d->n || d->drazin_index < 1))
        return PINV_ERR_ARG;
    if (d->kind == PINV_OUTER_G && (!d->G || d->ldg < d->m)) return PINV_ERR_ARG;
    if (d->kind < PINV_MOORE_PENROSE || d->kind > PINV_DRAZIN_NORMAL) return PINV_ERR_ARG;
    if (!(d->alpha >= 0.0) || !std::isfinite(d->alpha)) return PINV_ERR_ARG;
    if (!(d->tol >= 0.0)) return PINV_ERR_ARG;
    if (d->stop != PINV_STOP_REL_FRO && d->stop != PINV_STOP_PAPER && d->stop != PINV_STOP_ORDER18)
        return PINV_ERR_ARG;
    if (d->max_iter < 0 || d->max_iter > PINV_HISTORY) return PINV_ERR_ARG;
    if (d->prec != PINV_PREC_FP64 && d->prec != PINV_PREC_MIXED_BF16 && d->prec != PINV_PREC_FP32 &&
        d->prec != PINV_PREC_FP64_TC && d->prec != PINV_PREC_BF16_FP32 && d->prec != PINV_PREC_FP32_REFINE)
        return PINV_ERR_ARG;
    // the refinement steps end with the finish (its projection removes the
    // first-order rounding that order-2 steps do not contract)
    if (d->prec == PINV_PREC_FP32_REFINE && d->finish != PINV_FINISH_CLEAN) return PINV_ERR_ARG;
    // ... and only the Moore-Penrose and Drazin finishes remove the FP32-class
    // rounding outside the range (measured on a weighted Moore-Penrose problem
    // through G: 3.9e-6 after the X A X finish, where FP64-class products stay
    // within 1e-9)
    if (d->prec == PINV_PREC_FP32_REFINE && d->kind != PINV_MOORE_PENROSE && d->kind != PINV_DRAZIN)
        return PINV_ERR_ARG;
    if (d->variant != PINV_VARIANT_PLAIN && d->variant != PINV_VARIANT_STABILIZED) return PINV_ERR_ARG;
    if (d->finish != PINV_FINISH_NONE && d->finish != PINV_FINISH_CLEAN) return PINV_ERR_ARG;
    // BF16/FP32-class loops leave rounding in the block the iteration does not
    // contract when m != n (Theorem 6.2: E12 or E21 persists); only the finish
    // step removes it, so low-precision schedules on rectangular problems need it
    if ((d->prec == PINV_PREC_MIXED_BF16 || d->prec == PINV_PREC_FP32 || d->prec == PINV_PREC_BF16_FP32) &&
        d->m != d->n &&
        d->finish != PINV_FINISH_CLEAN)
        return PINV_ERR_ARG;
    return PINV_OK;
}

// Largest side of a single solve whose loops are replayed from cached graphs.
constexpr int kReplayMaxDim = 512;

int setup_context(pinv_handle* h, const pinv_desc* d, cudaStream_t st, Ctx& c, bool cplx = false) {
    c.h = h;
    c.st = st;
    c.cplx = cplx;
    c.m = cplx ? 2 * d->m : d->m;   // complex: the real embedding is 2m x 2n
    c.n = cplx ? 2 * d->n : d->n;
    c.left = c.m > c.n;  // residual on the smaller side; the paper's right form when m <= n
    c.s = c.left ? c.n : c.m;
    c.c = pm_coefficients();
    const bool drazin = d->kind == PINV_DRAZIN || d->kind == PINV_DRAZIN_NORMAL;
    const bool host = d->host_buffers != 0;
    const bool check = d->check != 0 || d->finish == PINV_FINISH_CLEAN;
    c.replay = !c.profile && std::max(c.m, c.n) <= kReplayMaxDim;
    const bool own_a = host || c.replay || cplx;   // A (and G) live in the workspace
    size_t bytes = workspace_bytes(c.m, c.n, drazin, own_a, check, d->prec);
    int rc = ensure_workspace(h, bytes);
    if (rc) return rc;
    carve(c, drazin, own_a, check, d->prec);
    c.prec_k = d->prec == PINV_PREC_FP64 ? 0 : TC_FP64;
    c.symmetric = !cplx && iterates_symmetric(d);
    if (cplx) {
        // A (m x n complex) -> E(A) in the workspace; host inputs are staged in
        // the half-step and pong iterates, which are free until the first loop
        const double* Z = d->A;
        int ldz = d->lda;
        if (host) {
            CK(cudaMemcpy2DAsync(c.X[2], 2 * sizeof(double) * d->n, d->A, 2 * sizeof(double) * d->lda,
                                 2 * sizeof(double) * d->n, d->m, cudaMemcpyHostToDevice, st));
            Z = c.X[2];
            ldz = d->n;
        }
        complex_embed(d->m, d->n, Z, ldz, c.Ad, c.n, st);
        ++c.kernels;
        c.A = c.Ad;
        c.lda = c.n;
        if (d->kind == PINV_OUTER_G) {   // G (n x m complex) -> E(G), 2n x 2m
            const double* Zg = d->G;
            int ldg = d->ldg;
            if (host) {
                CK(cudaMemcpy2DAsync(c.X[1], 2 * sizeof(double) * d->m, d->G, 2 * sizeof(double) * d->ldg,
                                     2 * sizeof(double) * d->m, d->n, cudaMemcpyHostToDevice, st));
                Zg = c.X[1];
                ldg = d->m;
            }
            complex_embed(d->n, d->m, Zg, ldg, c.Gd, c.m, st);
            ++c.kernels;
        }
        return PINV_OK;
    }
    if (host) {
        CK(cudaMemcpy2DAsync(c.Ad, sizeof(double) * d->n, d->A, sizeof(double) * d->lda,
                             sizeof(double) * d->n, d->m, cudaMemcpyHostToDevice, st));
        c.A = c.Ad;
        c.lda = d->n;
        if (d->kind == PINV_OUTER_G) {
            CK(cudaMemcpy2DAsync(c.Gd, sizeof(double) * d->m, d->G, sizeof(double) * d->ldg,
                                 sizeof(double) * d->m, d->n, cudaMemcpyHostToDevice, st));
        }
    } else if (c.replay) {   // device copy, so the cached loop graph never refers to caller memory
        CK(cudaMemcpy2DAsync(c.Ad, sizeof(double) * d->n, d->A, sizeof(double) * d->lda,
                             sizeof(double) * d->n, d->m, cudaMemcpyDeviceToDevice, st));
        c.A = c.Ad;
        c.lda = d->n;
    } else {
        c.A = d->A;
        c.lda = d->lda;
    }
    return PINV_OK;
}

// X0 = alpha G (Section 4) into c.X[0]; returns alpha used via *alpha.
int initial_value(Ctx& c, const pinv_desc* d, double* alpha) {
    const int m = c.m, n = c.n;
    double a = d->alpha;
    if (d->kind == PINV_DRAZIN || d->kind == PINV_DRAZIN_NORMAL) {
        const int l = d->drazin_index;
        // A^l by l - 1 products
        scale_copy(n, n, c.A, c.lda, 1.0, c.Al, n, c.st);
        ++c.kernels;
        for (int i = 1; i < l; ++i) {
            gemm(c, n, n, n, c.Al, n, false, c.A, c.lda, false, epi1(term(c.sq[0], n, 1)));
            scale_copy(n, n, c.sq[0], n, 1.0, c.Al, n, c.st);
            ++c.kernels;
        }
        if (d->kind == PINV_DRAZIN_NORMAL) {
            // G = A^l (A^{2l+1})^T A^l: A^{l+1} = A^l A, A^{2l+1} = A^{l+1} A^l,
            // W = (A^{2l+1})^T A^l, G = A^l W   (sq[0..2] as temporaries)
            double *Al1 = c.sq[0], *A2 = c.sq[1], *Wm = c.sq[2];
            gemm(c, n, n, n, c.Al, n, false, c.A, c.lda, false, epi1(term(Al1, n, 1)));
            gemm(c, n, n, n, Al1, n, false, c.Al, n, false, epi1(term(A2, n, 1)));
            gemm(c, n, n, n, A2, n, true, c.Al, n, false, epi1(term(Wm, n, 1)));
            gemm(c, n, n, n, c.Al, n, false, Wm, n, false, epi1(term(c.X[1], m, 1)));   // G
            if (a == 0.0) {   // 1 / sqrt(||GA||_1 ||GA||_inf) <= 1 / ||GA||_2
                gemm(c, n, n, n, c.X[1], m, false, c.A, c.lda, false, epi1(term(A2, n, 1)));
                if (c.cplx) complex_norms_1_inf(n / 2, n / 2, A2, n, c.h->dsmall, c.red, c.st);
                else        norms_1_inf(n, n, A2, n, c.h->dsmall, c.red, c.st);
                c.kernels += 4;
                CK(cudaMemcpyAsync(c.h->pinned, c.h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
                CK(cudaStreamSynchronize(c.st));
                const double pr = c.h->pinned[0] * c.h->pinned[1];
                if (!std::isfinite(pr)) return PINV_ERR_NONFINITE;
                a = pr > 0.0 ? 1.0 / std::sqrt(pr) : 1.0;   // GA = 0: X0 = 0 for every alpha
            }
            scale_copy(n, n, c.X[1], m, a, c.X[0], m, c.st);
            ++c.kernels;
            *alpha = a;
            return PINV_OK;
        }
        if (a == 0.0) {  // alpha = 1 / Tr(A^{l+1}) = 1 / sum_ij (A^l)_ij A_ji
            trace_of_product(n, c.Al, n, c.A, c.lda, c.h->dsmall, c.red, c.st);
            c.kernels += 2;
            CK(cudaMemcpyAsync(c.h->pinned, c.h->dsmall, sizeof(double), cudaMemcpyDeviceToHost, c.st));
            CK(cudaStreamSynchronize(c.st));
            // complex: Tr E(A^{l+1}) = 2 Re Tr(A^{l+1}); alpha = 1 / Re Tr(A^{l+1})
            const double tr = c.cplx ? 0.5 * c.h->pinned[0] : c.h->pinned[0];
            if (!(tr > 0.0) || !std::isfinite(tr)) return PINV_ERR_ARG;
            a = 1.0 / tr;
        }
        scale_copy(n, n, c.Al, n, a, c.X[0], m, c.st);
        ++c.kernels;
    } else {
        const bool own_g = d->host_buffers || c.cplx;
        const double* G = own_g ? c.Gd : d->G;
        const int ldg = own_g ? m : d->ldg;
        if (a == 0.0) {
            // Moore-Penrose: 1 / (||A||_1 ||A||_inf) (Section 4).  General G:
            // 1 / sqrt(||P||_1 ||P||_inf), P = GA (left side) or AG, the smaller
            // square with the nonzero eigenvalues of GA, whose spectral radius
            // it bounds.  Complex moduli for complex matrices.
            const double* N1 = c.A;
            int r = m, cols = n, ld = c.lda;
            if (d->kind == PINV_OUTER_G) {
                double* P = c.sq[0];
                if (c.left) gemm(c, n, n, m, G, ldg, false, c.A, c.lda, false, epi1(term(P, n, 1)));
                else        gemm(c, m, m, n, c.A, c.lda, false, G, ldg, false, epi1(term(P, m, 1)));
                N1 = P;
                r = cols = ld = c.s;
            }
            if (c.cplx) complex_norms_1_inf(r / 2, cols / 2, N1, ld, c.h->dsmall, c.red, c.st);
            else        norms_1_inf(r, cols, N1, ld, c.h->dsmall, c.red, c.st);
            c.kernels += 4;
            CK(cudaMemcpyAsync(c.h->pinned, c.h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
            CK(cudaStreamSynchronize(c.st));
            const double p = c.h->pinned[0] * c.h->pinned[1];
            if (!std::isfinite(p)) return PINV_ERR_NONFINITE;
            // A = 0 (or GA = 0): X0 = 0 for every alpha and X = 0 is the answer;
            // take alpha = 1 as a batched group does
            a = !(p > 0.0) ? 1.0 : (d->kind == PINV_OUTER_G ? 1.0 / std::sqrt(p) : 1.0 / p);
        }
        if (d->kind == PINV_MOORE_PENROSE) {
            transpose_scale(m, n, c.A, c.lda, a, c.X[0], m, c.st);
            ++c.kernels;
        } else {
            scale_copy(n, m, G, ldg, a, c.X[0], m, c.st);
            ++c.kernels;
        }
    }
    *alpha = a;
    return PINV_OK;
}

// A loop that leaves X unchanged has reached the fixed point of the iteration
// (X_{k+1} = X_k); its measure is 0 under every rule (the relative rule would
// otherwise be 0/0 when X = 0, e.g. A = 0 or G = 0, where X = 0 is the answer).
double stop_measure(const pinv_desc* d, double dx2, double x2, int k, double alpha) {
    if (dx2 == 0.0) return 0.0;
    const double dx = std::sqrt(dx2);
    if (d->stop == PINV_STOP_PAPER) return dx / (std::pow(18.0, k) * alpha);
    return x2 > 0 ? dx / std::sqrt(x2) : INFINITY;
}

// Small solves are bound by launch and host overhead: their loop (seven or nine
// products, the norm reduction and the readback) runs as one cached graph.
// The stop rule of a plain loop at one precision, on the device (one thread):
// the same arithmetic and decisions as the host loop in solve_one, reading the
// loop's reduced norms.  It always ends the WHILE loop by k = max_iter, so the
// device loop terminates whatever the data.
__global__ void loop_decide_kernel(cudaGraphConditionalHandle cond, const double* norms, const int* derr,
                                   DeviceLoopState* st) {
    if (threadIdx.x != 0) return;
    const int k = st->k;
    const double dx2 = norms[0], x2 = norms[1];
    double e;
    if (dx2 == 0.0) {
        e = 0.0;
    } else if (st->stop_mode == PINV_STOP_PAPER) {
        double p18 = 1.0;
        for (int i = 0; i < k; ++i) p18 *= 18.0;
        e = sqrt(dx2) / (p18 * st->alpha);
    } else {
        e = x2 > 0 ? sqrt(dx2) / sqrt(x2) : INFINITY;
    }
    if (k < PINV_HISTORY) st->history[k] = e;
    st->loops_run = k + 1;
    int stop = 0, copy = 0;
    if (*derr) {
        st->status = PINV_ERR_TIMEOUT; stop = 1;
    } else if (!isfinite(e)) {
        st->status = PINV_ERR_NONFINITE; st->iters = k; stop = 1;
    } else if (e < st->tol) {
        st->status = PINV_OK; st->reason = 0; st->iters = k + 1; st->rel_step = e; stop = 1; copy = 1;
    } else {
        const double prev = st->prev;
        const bool stalled = k >= 1 && prev < 1e-3 && e >= prev * prev;
        const double rel = dx2 == 0.0 ? 0.0 : (x2 > 0 ? sqrt(dx2 / x2) : INFINITY);
        if (stalled) {
            st->status = PINV_OK; st->reason = 1; st->iters = k; st->rel_step = prev; stop = 1;
        } else if (rel > 1e3 && k > 0) {
            st->status = PINV_ERR_DIVERGED; st->iters = k; stop = 1;
        } else {
            st->prev2 = prev;
            st->prev = e;
            st->rel_step = e;
            st->iters = k + 1;
            copy = 1;
            if (k + 1 >= st->max_iter) { st->status = PINV_ERR_MAXITER; st->reason = 2; stop = 1; }
        }
    }
    st->k = k + 1;
    st->copy = copy;
    cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

// X0 <- X1 when the decision kept the new iterate (device loop ping-pong).
__global__ void loop_copy_kernel(const DeviceLoopState* st, const double* src, double* dst, size_t count) {
    if (!st->copy) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

constexpr int kDeviceLoopUnavailable = 1000;   // not a PINV code: fall back to the host loop

// Whole solve loop on the device for small plain solves at one precision: a
// graph with a WHILE node whose body is the loop, the norm reduction, the stop
// decision and the ping-pong copy; one launch and one readback per solve.
int device_loop(Ctx& c, const pinv_desc* d, double alpha, int max_iter, pinv_info* info) {
    pinv_handle* h = c.h;
    if (!h->dstate) {
        CK(cudaMalloc((void**)&h->dstate, sizeof(DeviceLoopState)));
        CK(cudaMallocHost((void**)&h->hstate, sizeof(DeviceLoopState)));
    }
    std::vector<long long> key = {-1, c.m, c.n, c.left, c.symmetric, c.cplx, c.prec_k, h->tc_crossover,
                                  (long long)c.A, c.lda, (long long)c.X[0], (long long)c.X[1],
                                  (long long)c.sq[0], (long long)c.partials, (long long)c.tcws,
                                  (long long)c.tcws_bytes};
    pinv_handle::LoopGraph* lg = nullptr;
    for (auto& g : h->loop_graphs)
        if (g.key == key) { lg = &g; break; }
    if (!lg) {
        if (!h->capture_stream) CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
        if (h->loop_graphs.size() >= 32) {
            cudaGraphExecDestroy(h->loop_graphs.front().exec);
            h->loop_graphs.erase(h->loop_graphs.begin());
        }
        cudaGraph_t graph = nullptr;
        CK(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle cond;
        cudaGraphNodeParams np = {};
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = cond;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
        }
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            std::fprintf(stderr, "pinv: device loop graph: %s (host loop used)\n", cudaGetErrorString(e));
            h->device_loop_off = true;
            return kDeviceLoopUnavailable;
        }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        cudaStream_t user = c.st;
        c.st = h->capture_stream;
        const int k0 = c.kernels, g0 = c.gemms;
        e = cudaStreamBeginCaptureToGraph(c.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        int parts = -1;
        if (e == cudaSuccess) {
            parts = pm_loop_f64(c, c.X[0], c.X[1]);
            if (parts >= 0) {
                reduce_pairs(c.partials, parts, h->dsmall, c.st);
                loop_decide_kernel<<<1, 32, 0, c.st>>>(cond, h->dsmall, h->derr, h->dstate);
                loop_copy_kernel<<<64, 256, 0, c.st>>>(h->dstate, c.X[1], c.X[0], (size_t)c.n * c.m);
            }
            cudaGraph_t captured = nullptr;
            e = cudaStreamEndCapture(c.st, &captured);
        }
        c.st = user;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess && parts >= 0) e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess || parts < 0) {
            std::fprintf(stderr, "pinv: device loop graph: %s (host loop used)\n", cudaGetErrorString(e));
            c.kernels = k0;
            c.gemms = g0;
            cudaGetLastError();
            h->device_loop_off = true;
            return kDeviceLoopUnavailable;
        }
        pinv_handle::LoopGraph g;
        g.key = key;
        g.exec = exec;
        g.kernels = c.kernels - k0 + 3;   // + reduction, decision, copy
        g.gemms = c.gemms - g0;
        c.kernels = k0;
        c.gemms = g0;
        h->loop_graphs.push_back(std::move(g));
        lg = &h->loop_graphs.back();
    }
    DeviceLoopState& hs = *h->hstate;
    std::memset(&hs, 0, sizeof(hs));
    hs.max_iter = max_iter;
    hs.stop_mode = d->stop;
    hs.alpha = alpha;
    hs.tol = d->tol;
    hs.prev = hs.prev2 = INFINITY;
    hs.status = PINV_ERR_MAXITER;
    hs.reason = 2;
    CK(cudaMemcpyAsync(h->dstate, &hs, sizeof(hs), cudaMemcpyHostToDevice, c.st));
    CK(cudaGraphLaunch(lg->exec, c.st));
    CK(cudaMemcpyAsync(&hs, h->dstate, sizeof(hs), cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    c.kernels += lg->kernels * hs.loops_run;
    c.gemms += lg->gemms * hs.loops_run;
    info->loops_run = hs.loops_run;
    info->iters = hs.iters;
    info->rel_step = hs.rel_step;
    info->stop_reason = hs.reason;
    for (int k = 0; k < std::min(hs.loops_run, PINV_HISTORY); ++k) {
        info->history[k] = hs.history[k];
        info->precision[k] = (signed char)c.prec_k;
    }
    if (hs.status == PINV_ERR_TIMEOUT) {
        std::fprintf(stderr, "pinv: tensor-core kernel wait timed out\n");
        cudaMemsetAsync(h->derr, 0, sizeof(int), c.st);
    }
    return hs.status;
}

int replay_loop(Ctx& c, int cur, bool stab, double* dx2, double* x2) {
    pinv_handle* h = c.h;
    const double* Xk = c.X[cur];
    double* Xn = c.X[cur ^ 1];
    std::vector<long long> key = {c.m, c.n, c.left, c.symmetric, c.cplx, c.prec_k, stab, h->tc_crossover,
                                  (long long)c.A, c.lda, (long long)Xk, (long long)Xn, (long long)c.X[2],
                                  (long long)c.sq[0], (long long)c.partials, (long long)c.tcws,
                                  (long long)c.tcws_bytes};
    pinv_handle::LoopGraph* lg = nullptr;
    for (auto& g : h->loop_graphs)
        if (g.key == key) { lg = &g; break; }
    if (!lg) {
        if (!h->capture_stream) CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
        if (h->loop_graphs.size() >= 32) {   // bounded cache: drop the oldest
            cudaGraphExecDestroy(h->loop_graphs.front().exec);
            h->loop_graphs.erase(h->loop_graphs.begin());
        }
        cudaStream_t user = c.st;
        c.st = h->capture_stream;
        const int k0 = c.kernels, g0 = c.gemms;
        CK(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal));
        int parts = pm_loop_f64(c, Xk, stab ? c.X[2] : Xn);
        if (stab && parts >= 0) parts = stabilise_f64(c, c.X[2], Xk, Xn);
        if (parts >= 0) {
            reduce_pairs(c.partials, parts, h->dsmall, c.st);
            cudaMemcpyAsync(h->pinned, h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st);
            cudaMemcpyAsync(h->pinned + 2, h->derr, sizeof(int), cudaMemcpyDeviceToHost, c.st);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(c.st, &graph);
        c.st = user;
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = (parts >= 0 && ce == cudaSuccess && graph) ? cudaGraphInstantiate(&exec, graph, 0)
                                                                          : cudaErrorUnknown;
        if (graph) cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            std::fprintf(stderr, "pinv: loop graph capture failed (%s)\n", cudaGetErrorString(ce != cudaSuccess ? ce : ie));
            return PINV_ERR_CUDA;
        }
        pinv_handle::LoopGraph g;
        g.key = key;
        g.exec = exec;
        g.kernels = c.kernels - k0 + 1;   // + the reduction
        g.gemms = c.gemms - g0;
        c.kernels = k0;
        c.gemms = g0;
        h->loop_graphs.push_back(std::move(g));
        lg = &h->loop_graphs.back();
    }
    CK(cudaGraphLaunch(lg->exec, c.st));
    c.kernels += lg->kernels;
    c.gemms += lg->gemms;
    CK(cudaStreamSynchronize(c.st));
    *dx2 = h->pinned[0];
    *x2 = h->pinned[1];
    int derr;
    std::memcpy(&derr, h->pinned + 2, sizeof(int));
    if (derr) {
        std::fprintf(stderr, "pinv: tensor-core kernel wait timed out (code %d)\n", derr);
        cudaMemsetAsync(h->derr, 0, sizeof(int), c.st);
        return PINV_ERR_TIMEOUT;
    }
    return PINV_OK;
}

// The result Xfinal to the caller's X (device or host, real or complex; `spare`
// is a free iterate buffer for staging), then the call's counters into info.
int copy_out(Ctx& c, const pinv_desc* d, const double* Xfinal, double* spare, pinv_info* info,
             std::chrono::steady_clock::time_point t0) {
    cudaStream_t st = c.st;
    if (c.cplx) {   // X (n x m complex) from the left half of E(X)
        if (d->host_buffers) {
            complex_extract(d->n, d->m, Xfinal, c.m, spare, d->m, st);
            CK(cudaMemcpy2DAsync(d->X, 2 * sizeof(double) * d->ldx, spare, 2 * sizeof(double) * d->m,
                                 2 * sizeof(double) * d->m, d->n, cudaMemcpyDeviceToHost, st));
        } else {
            complex_extract(d->n, d->m, Xfinal, c.m, d->X, d->ldx, st);
        }
        ++c.kernels;
    } else if (d->host_buffers) {
        CK(cudaMemcpy2DAsync(d->X, sizeof(double) * d->ldx, Xfinal, sizeof(double) * c.m,
                             sizeof(double) * c.m, c.n, cudaMemcpyDeviceToHost, st));
    } else {
        CK(cudaMemcpy2DAsync(d->X, sizeof(double) * d->ldx, Xfinal, sizeof(double) * c.m,
                             sizeof(double) * c.m, c.n, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    prof_harvest(c);
    info->gemms = c.gemms;
    info->kernels = c.kernels;
    info->gemm_ms = c.gemm_ms;
    info->gemm_flops = c.gemm_flops;
    info->tensor_flops = c.tensor_flops;
    info->ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return PINV_OK;
}

// Approximate-inverse preconditioner (Section 8, Example 3): `loops` loops of
// Eq. PM from the Jacobi X0 = alpha diag(1/a_ii) (Eq. choice3), each followed
// by the chop when chop > 0.  No stop rule: the loop count is the request.
int precond_one(pinv_handle* h, const pinv_precond_desc* p, cudaStream_t st, pinv_info* info) {
    auto t0 = std::chrono::steady_clock::now();
    std::memset(info, 0, sizeof(*info));
    if (!p || p->n < 1 || !p->A || !p->X || p->lda < p->n || p->ldx < p->n || p->loops < 1 ||
        p->loops > PINV_HISTORY || !(p->alpha >= 0.0) || !std::isfinite(p->alpha) || !(p->chop >= 0.0) ||
        !std::isfinite(p->chop))
        return info->status = PINV_ERR_ARG;
    int level;
    switch (p->prec) {
        case PINV_PREC_FP64: level = 0; break;
        case PINV_PREC_FP64_TC: level = TC_FP64; break;
        case PINV_PREC_FP32: level = TC_FP32; break;
        case PINV_PREC_MIXED_BF16:
        case PINV_PREC_BF16_FP32: level = TC_BF16; break;
        default: return info->status = PINV_ERR_ARG;
    }
    pinv_desc d{};
    d.m = d.n = p->n;
    d.A = p->A;
    d.lda = p->lda;
    d.X = p->X;
    d.ldx = p->ldx;
    d.kind = PINV_MOORE_PENROSE;   // no G to stage
    d.prec = p->prec == PINV_PREC_FP64 ? PINV_PREC_FP64 : PINV_PREC_FP64_TC;   // workspace for any class
    d.host_buffers = p->host_buffers;
    Ctx c{};
    c.profile = p->profile != 0;
    const bool cplx = p->complex_matrix != 0;
    int rc = setup_context(h, &d, st, c, cplx);
    if (rc) return info->status = rc;
    const int n = c.n;   // 2 p->n for a complex matrix
    CK(cudaMemsetAsync(c.X[0], 0, sizeof(double) * (size_t)n * n, st));
    jacobi_x0(p->n, c.A, c.lda, p->alpha > 0 ? p->alpha : 1.0, c.X[0], n, cplx, h->dsmall, st);
    ++c.kernels;
    CK(cudaMemcpyAsync(h->pinned, h->dsmall, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->pinned[0] != 0.0) return info->status = PINV_ERR_ARG;   // a zero diagonal entry
    info->alpha = p->alpha > 0 ? p->alpha : 1.0;
    c.prec_k = level;
    int cur = 0;
    for (int k = 0; k < p->loops; ++k) {
        const int parts = pm_loop_f64(c, c.X[cur], c.X[cur ^ 1]);
        if (parts < 0) return info->status = PINV_ERR_CUDA;
        if (p->chop > 0) {
            chop(n, n, c.X[cur ^ 1], n, p->chop, st);
            ++c.kernels;
        }
        double dx2, x2;
        rc = read_norms(c, parts, &dx2, &x2);
        if (rc) return info->status = rc;
        const double e = dx2 == 0.0 ? 0.0 : (x2 > 0 ? std::sqrt(dx2 / x2) : INFINITY);
        info->history[k] = e;
        info->precision[k] = (signed char)level;
        info->loops_run = info->iters = k + 1;
        info->rel_step = e;
        cur ^= 1;
        if (!std::isfinite(e)) return info->status = PINV_ERR_NONFINITE;
    }
    info->side = c.left ? 1 : 0;
    rc = copy_out(c, &d, c.X[cur], c.X[cur ^ 1], info, t0);
    return info->status = rc;
}

// The refinement of PINV_PREC_FP32_REFINE, after its last FP32-class loop
// (X[cur] holds that loop's iterate, X[cur ^ 1] is free):
//  1. X <- X A X in FP32 class (Section 7's stabilising product; XAX = X holds
//     for every outer inverse, Eq. 1): it removes the loop's first-order
//     rounding outside R(X) and N(X), which an order-2 step would double
//     (order p multiplies the blocks the iteration does not contract by p,
//     Theorem 6.2);
//  2. order-2 steps X <- X + (I - XA) X (Eq. hyper, p = 2): the step's
//     relative change e_j bounds the error of its input in the range, and each
//     step squares that error, so the input error of step j is also below
//     e_{j-1}^2.  The steps stop after the first FP64-class one with
//     min(e_j, e_{j-1}^2) < 1e-5: its output's range error is below the square
//     of that.  (On a Drazin problem e_j keeps a part that does not contract,
//     from the block of the nilpotent part that the finish removes; there the
//     e_{j-1}^2 bound ends the steps.)  The first step runs in FP32 class: its
//     input error (~1e-3 after the loop) squared is still far above its own
//     rounding, which the next, FP64-class step squares away in turn.
// The kept iterate ends in X[cur].  Returns PINV_OK, or an error status.
constexpr int kRefineMaxSteps = 16;   // from an error near 1, eleven steps reach 1e-9
constexpr double kRefineTol = 1e-5;

int refine_steps(Ctx& c, int& cur, pinv_info* info, int* reason) {
    c.prec_k = TC_FP32;
    int parts = stabilise_f64(c, c.X[cur], c.X[cur ^ 1], c.X[2]);
    if (parts < 0) return PINV_ERR_CUDA;
    ++info->stabilized_loops;
    const double* src = c.X[2];
    double prev_e = INFINITY;
    for (int j = 0; j < kRefineMaxSteps; ++j) {
        c.prec_k = j == 0 ? TC_FP32 : TC_FP64;
        parts = ns_step_f64(c, src, c.X[cur ^ 1]);
        if (parts < 0) return PINV_ERR_CUDA;
        double dx2, x2;
        int rc = read_norms(c, parts, &dx2, &x2);
        if (rc) return rc;
        cur ^= 1;
        src = c.X[cur];
        const double e = dx2 == 0.0 ? 0.0 : (x2 > 0 ? std::sqrt(dx2 / x2) : INFINITY);
        const int k = info->loops_run++;
        if (k < PINV_HISTORY) {
            info->history[k] = e;
            info->precision[k] = j == 0 ? 5 : 6;
        }
        ++info->iters;
        info->rel_step = e;
        if (!std::isfinite(e)) return PINV_ERR_NONFINITE;
        if (e > 1e3) return PINV_ERR_DIVERGED;
        if (j > 0 && std::min(e, prev_e * prev_e) < kRefineTol) { *reason = 0; return PINV_OK; }
        prev_e = e;
    }
    *reason = 2;
    return PINV_ERR_MAXITER;
}

int solve_one(pinv_handle* h, const pinv_desc* d, cudaStream_t st, pinv_info* info, bool cplx = false) {
    auto t0 = std::chrono::steady_clock::now();
    std::memset(info, 0, sizeof(*info));
    int rc = validate(d);
    if (!rc && cplx && d->symmetric) rc = PINV_ERR_ARG;
    if (rc) return info->status = rc;
    Ctx c{};
    c.profile = d->profile != 0;
    rc = setup_context(h, d, st, c, cplx);
    if (rc) return info->status = rc;
    info->side = c.left ? 1 : 0;
    double alpha = 0.0;
    rc = initial_value(c, d, &alpha);
    if (rc) return info->status = rc;
    info->alpha = alpha;

    const int max_iter = d->max_iter ? d->max_iter : 100;
    const double switch_tol = d->switch_tol > 0 ? d->switch_tol : 1e-3;
    // small problems replay each loop from a cached graph (the matrix is in the
    // workspace then, so the graph serves any later solve of the same shape)
    const bool replay = c.replay;
    const double floor_guard = 1e-3;
    int cur = 0;              // X[cur] = X_k
    double prev = INFINITY;
    bool stabilise = false;
    int status = PINV_ERR_MAXITER, reason = 2;
    // the precision of the last loops (and of the stop rule): native FP64, the
    // FP64-class slice engine, or FP32-class for the FP32-finished schedule
    const int fp64_class = d->prec == PINV_PREC_FP64 ? 0 : (d->prec == PINV_PREC_BF16_FP32 ? TC_FP32 : TC_FP64);
    // Precision schedule (next_level): the class only rises, BF16 -> FP32-class
    // -> final class; the stop rule and the stabilising product use final-class
    // loops only.
    const bool refine = d->prec == PINV_PREC_FP32_REFINE;
    int level = (d->prec == PINV_PREC_MIXED_BF16 || d->prec == PINV_PREC_BF16_FP32)
                    ? TC_BF16 : ((d->prec == PINV_PREC_FP32 || refine) ? TC_FP32 : fp64_class);
    bool refine_now = false;  // the FP32-class loops of the refine schedule have ended
    int prev_prec = -1;
    double prev_rel = INFINITY;   // relative step of the last loop (schedule input)
    bool bf16_ran = false;
    // Small plain solves at one precision run the whole loop on the device (a
    // graph WHILE node with the stop rule in a kernel): one launch per solve.
    bool on_device = replay && !h->device_loop_off && d->variant == PINV_VARIANT_PLAIN && level == fp64_class &&
                     max_iter <= 1000;
    if (on_device) {
        c.prec_k = level;
        status = device_loop(c, d, alpha, max_iter, info);
        if (status == kDeviceLoopUnavailable) {
            on_device = false;
            status = PINV_ERR_MAXITER;
        } else {
            if (status == PINV_ERR_CUDA || status == PINV_ERR_TIMEOUT) return info->status = status;
            reason = info->stop_reason;
            cur = 0;   // the kept iterate is in X[0]
        }
    }
    for (int k = 0; !on_device && k < max_iter; ++k) {
        const double* Xk = c.X[cur];
        double* Xn = c.X[cur ^ 1];
        int parts;
        // product class of loop k (the step of loop k-1 says how far from
        // convergence the iterate is; low precision only far from it)
        level = next_level(level, prev_prec, fp64_class, prev_rel);
        const int prec_k = level;
        c.prec_k = prec_k;
        if (prec_k == TC_BF16) bf16_ran = true;
        // the stabilising product runs in final-class loops only
        const bool stab_now = stabilise && prec_k == fp64_class;
        double dx2, x2;
        if (stab_now) ++info->stabilized_loops;
        if (replay) {
            rc = replay_loop(c, cur, stab_now, &dx2, &x2);
            if (rc) return info->status = rc;
        } else {
            double* target = stab_now ? c.X[2] : Xn;
            parts = pm_loop_f64(c, Xk, target);
            if (stab_now) parts = stabilise_f64(c, c.X[2], Xk, Xn);
            if (parts < 0) return info->status = PINV_ERR_CUDA;
            rc = read_norms(c, parts, &dx2, &x2);
            if (rc) return info->status = rc;
        }
        const double e = stop_measure(d, dx2, x2, k, alpha);
        info->loops_run = k + 1;
        if (k < PINV_HISTORY) {
            info->history[k] = e;
            info->precision[k] = (signed char)(prec_k == 0 ? 0 : prec_k);
        }
        if (!std::isfinite(e)) { status = PINV_ERR_NONFINITE; info->iters = k; break; }
        // ORDER18: the threshold is trusted in final-precision loops only
        const bool tol_ok = d->stop != PINV_STOP_ORDER18 || prec_k == fp64_class;
        if (e < d->tol && tol_ok) { status = PINV_OK; reason = 0; cur ^= 1; info->iters = k + 1; info->rel_step = e; break; }
        // the stop rule compares two consecutive FP64-class loops only: the first
        // FP64-class step after lower-precision loops removes their noise
        const bool final_class = prec_k == fp64_class && prev_prec == fp64_class;
        const bool stalled = stab_now ? (e >= prev) : (prev < floor_guard && e >= prev * prev);
        if (stalled && final_class) { status = PINV_OK; reason = 1; info->iters = k; info->rel_step = prev; break; }
        // divergence guard on the relative step: a convergent loop grows X by at
        // most a factor 18 (|p(r)| <= 18 for |r| <= 1)
        const double rel = dx2 == 0.0 ? 0.0 : (x2 > 0 ? std::sqrt(dx2 / x2) : INFINITY);
        if (rel > 1e3 && k > 0) { status = PINV_ERR_DIVERGED; info->iters = k; break; }
        // refine schedule: the first loop whose step is below 1 is one order-18
        // contraction from its limit; the order-2 refinement steps take it from there
        if (refine && rel < 1.0) { refine_now = true; cur ^= 1; info->iters = k + 1; info->rel_step = e; break; }
        if (d->variant == PINV_VARIANT_STABILIZED && e < switch_tol) stabilise = true;
        prev = e;
        prev_rel = rel;
        prev_prec = prec_k;
        info->rel_step = e;
        cur ^= 1;
        info->iters = k + 1;
    }
    if (refine_now) {
        status = refine_steps(c, cur, info, &reason);
        if (status == PINV_ERR_CUDA || status == PINV_ERR_TIMEOUT) return info->status = status;
    }
    info->stop_reason = reason;
    c.prec_k = fp64_class;   // the finish runs in the schedule's final class
    if (status == PINV_OK && d->finish == PINV_FINISH_CLEAN) {
        // projection, then one order-2 step (Theorems 6.2 / 7.1: the blocks the
        // loop does not contract are removed; the step squares the projection's
        // first-order rounding in the range block) -- or one order-18 loop
        // after BF16 loops
        cleanup_f64(c, d, c.X[cur], c.X[cur ^ 1]);
        int parts = !bf16_ran ? ns_step_f64(c, c.X[cur ^ 1], c.X[cur]) : pm_loop_f64(c, c.X[cur ^ 1], c.X[cur]);
        if (parts < 0) return info->status = PINV_ERR_CUDA;
    }
    const double* Xfinal = c.X[cur];
    if (status == PINV_OK && d->check) {
        rc = residual_checks(c, d, Xfinal, info);
        if (rc) return info->status = rc;
    }
    rc = copy_out(c, d, Xfinal, c.X[cur ^ 1], info, t0);
    return info->status = rc ? rc : status;
}


// ------------------------------------------------------------------ batched groups
// A group is a bucket of independent problems padded to one shape (zero rows
// and columns: the padded block of R is exactly I and the padded rows of X stay
// exactly 0, so every instance's iterate is its own problem's iterate).  Each
// instance owns one fixed-size slab of the workspace (A, three iterates, the
// seven squares, the two large squares), so every batched launch addresses
// instance b at +b*stride.  The group runs the chain of Eq. PM for all its
// instances in lockstep on its own stream; the stop rule is applied per
// instance on the host and an instance's kept iterate is copied to its caller
// buffer the moment it stops.
struct Group {
    pinv_handle* h = nullptr;
    cudaStream_t st = nullptr;
    std::vector<pinv_desc> d;
    std::vector<pinv_info> info;
    int batch = 0, M = 0, N = 0, prec = 0, fp64_class = 0, level = 0, prev_prec = -1;
    bool left = false, stabilise = false, finish = false;
    bool stab_now = false;         // the loop in flight appends the stabilising product
    bool bf16_ran = false;         // some loop ran BF16 products (finish: order-18 loop)
    int k = 0, cur = 0, max_iter = 100;
    char* mem = nullptr;
    double* pinned = nullptr;      // norms [2 batch] then masks
    Ctx c{};
    InstanceRef *tabA = nullptr, *tabX = nullptr, *tabG = nullptr;
    int* dmask = nullptr;          // 2 x batch: copy from X[cur], copy from X[cur^1]
    double* dalpha = nullptr;
    double* dnorms = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<double> prev, prev_rel;
    std::vector<char> done;
    int parts = 0;
    int err = PINV_OK;
    bool in_flight = false;        // a loop has been issued and not completed
    bool serving = false;          // priority stream by size, SMs released per tile
    // one CUDA graph per (precision level, stabilised, ping-pong side): the loop
    // chain is captured the first time and replayed afterwards
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, int> graph_parts, graph_kernels;

    ~Group() { release(); }
    // Stream-ordered release: no device-wide synchronisation, so retiring a
    // group never waits for other groups' kernels.
    void release() {
        if (st) cudaStreamSynchronize(st);
        for (auto& g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
        if (mem) cudaFreeAsync(mem, st);
        if (pinned) h->pinned_blocks.push_back(pinned);
        if (ev) cudaEventDestroy(ev);
        if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
        mem = nullptr; pinned = nullptr; ev = nullptr; st = nullptr;
    }
    // copy-out masks in the pinned block, after the norms and the error word
    int* loop_mask() const { return (int*)((char*)pinned + sizeof(double) * 2 * batch + 64); }
    int* finish_mask() const { return loop_mask() + 2 * batch; }
    bool active() const {
        if (err) return false;
        for (int b = 0; b < batch; ++b)
            if (!done[b]) return true;
        return false;
    }
};

constexpr size_t kPinnedBlock = 64 * 1024;   // readback block of a group (batch <= 1024)

size_t slab_doubles(int M, int N, bool big2, bool g) {
    auto al = [](size_t x) { return (x + 31) & ~size_t(31); };   // 256-byte multiples
    const size_t s = std::min(M, N), big = std::max(M, N);
    size_t t = al((size_t)M * N) + 3 * al((size_t)N * M) + 7 * al(s * s);
    if (big2) t += 2 * al(big * big);
    if (g) t += al((size_t)N * M);
    return t;
}

size_t group_bytes(int batch, int M, int N, int prec, bool big2, bool g) {
    const size_t big = std::max(M, N);
    size_t b = sizeof(double) * slab_doubles(M, N, big2, g) * batch;
    b += align_up(sizeof(double) * 2 * partial_pairs_bound(big, big) * batch);   // partials
    b += align_up(sizeof(double) * 2 * 2 * 256);                      // reduction scratch
    b += 3 * align_up(sizeof(InstanceRef) * batch) + align_up(sizeof(int) * 2 * batch) +
         2 * align_up(sizeof(double) * 2 * batch);
    if (prec != PINV_PREC_FP64) b += align_up(tc_workspace_bytes((int)big, (int)big, (int)big, tc_mode(TC_FP64), batch));
    return b + 4096;
}

int group_begin_impl(Group& G) {
    pinv_handle* h = G.h;
    const pinv_desc& d0 = G.d[0];
    G.batch = (int)G.d.size();
    G.prec = d0.prec;
    G.fp64_class = d0.prec == PINV_PREC_FP64 ? 0 : (d0.prec == PINV_PREC_BF16_FP32 ? TC_FP32 : TC_FP64);
    G.level = (d0.prec == PINV_PREC_MIXED_BF16 || d0.prec == PINV_PREC_BF16_FP32)
                  ? TC_BF16 : (d0.prec == PINV_PREC_FP32 ? TC_FP32 : G.fp64_class);
    G.left = G.M > G.N;
    G.finish = d0.finish == PINV_FINISH_CLEAN;
    G.max_iter = 0;
    for (auto& x : G.d) G.max_iter = std::max(G.max_iter, x.max_iter ? x.max_iter : 100);
    const bool gk = d0.kind == PINV_OUTER_G;
    G.info.assign(G.batch, pinv_info{});
    G.prev.assign(G.batch, INFINITY);
    G.prev_rel.assign(G.batch, INFINITY);
    G.done.assign(G.batch, 0);
    if (G.serving) {
        // smaller problems on higher-priority streams: their CTAs are scheduled
        // first whenever an SM frees up
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        const int big = std::max(G.M, G.N);
        const int span = least - greatest;   // greatest is the numerically smallest
        int prio = big <= 512 ? greatest : (big <= 2048 ? greatest + span / 2 : least);
        CK(cudaStreamCreateWithPriority(&G.st, cudaStreamNonBlocking, prio));
    } else {
        CK(cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking));
    }
    CK(cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming));
    const size_t bytes = group_bytes(G.batch, G.M, G.N, G.prec, G.finish, gk);
    if (!h->pool_ready) {   // keep freed group memory in the stream-ordered pool
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        h->pool_ready = true;
    }
    CK(cudaMallocAsync((void**)&G.mem, bytes, G.st));
    // pinned block: norms (2 doubles per instance), the error word, then the
    // copy-out masks of the loops and, separately, of the finish
    const size_t pin_bytes = sizeof(double) * 2 * G.batch + 64 + 2 * sizeof(int) * 2 * G.batch;
    if (pin_bytes <= kPinnedBlock && !h->pinned_blocks.empty()) {
        G.pinned = (double*)h->pinned_blocks.back();
        h->pinned_blocks.pop_back();
    } else {
        CK(cudaMallocHost(&G.pinned, std::max(pin_bytes, kPinnedBlock)));
    }
    // carve
    char* p = G.mem;
    auto take = [&](size_t n) { char* q = p; p += align_up(n); return q; };
    const long long slab = (long long)slab_doubles(G.M, G.N, G.finish, gk);
    double* slabs = (double*)take(sizeof(double) * slab * G.batch);
    Ctx& c = G.c;
    c.h = h; c.st = G.st; c.m = G.M; c.n = G.N; c.left = G.left; c.s = G.left ? G.N : G.M;
    c.c = pm_coefficients();
    c.batch = G.batch; c.stride = slab;
    c.yield_sms = G.serving;
    c.symmetric = iterates_symmetric(&d0);
    {
        auto al = [](size_t x) { return (x + 31) & ~size_t(31); };
        const size_t s2 = (size_t)c.s * c.s, big = std::max(G.M, G.N);
        double* q = slabs;
        c.Ad = q; q += al((size_t)G.M * G.N);
        for (int i = 0; i < 3; ++i) { c.X[i] = q; q += al((size_t)G.N * G.M); }
        for (int i = 0; i < 7; ++i) { c.sq[i] = q; q += al(s2); }
        c.big[0] = c.big[1] = nullptr;
        if (G.finish) { c.big[0] = q; q += al(big * big); c.big[1] = q; q += al(big * big); }
        c.Gd = nullptr;
        if (gk) { c.Gd = q; q += al((size_t)G.N * G.M); }
        c.A = c.Ad; c.lda = G.N; c.Al = nullptr;
    }
    const size_t big = std::max(G.M, G.N);
    c.partials = (double*)take(sizeof(double) * 2 * partial_pairs_bound(big, big) * G.batch);
    c.red = (double*)take(sizeof(double) * 2 * 2 * 256);
    G.tabA = (InstanceRef*)take(sizeof(InstanceRef) * G.batch);
    G.tabX = (InstanceRef*)take(sizeof(InstanceRef) * G.batch);
    G.tabG = (InstanceRef*)take(sizeof(InstanceRef) * G.batch);
    G.dmask = (int*)take(sizeof(int) * 2 * G.batch);
    G.dalpha = (double*)take(sizeof(double) * 2 * G.batch);
    G.dnorms = (double*)take(sizeof(double) * 2 * G.batch);
    if (G.prec != PINV_PREC_FP64) {
        c.tcws_bytes = tc_workspace_bytes((int)big, (int)big, (int)big, tc_mode(TC_FP64), G.batch);
        c.tcws = take(c.tcws_bytes);
    }
    // instance tables and alphas
    std::vector<InstanceRef> ta(G.batch), tx(G.batch), tg(G.batch);
    std::vector<double> alpha(G.batch);
    for (int b = 0; b < G.batch; ++b) {
        const pinv_desc& x = G.d[b];
        ta[b] = InstanceRef{x.A, nullptr, x.m, x.n, x.lda, 0};
        tx[b] = InstanceRef{nullptr, x.X, x.n, x.m, x.ldx, 0};
        tg[b] = InstanceRef{x.G, nullptr, x.n, x.m, x.ldg, 0};
        alpha[b] = x.alpha;
    }
    CK(cudaMemcpyAsync(G.tabA, ta.data(), sizeof(InstanceRef) * G.batch, cudaMemcpyHostToDevice, G.st));
    CK(cudaMemcpyAsync(G.tabX, tx.data(), sizeof(InstanceRef) * G.batch, cudaMemcpyHostToDevice, G.st));
    CK(cudaMemcpyAsync(G.tabG, tg.data(), sizeof(InstanceRef) * G.batch, cudaMemcpyHostToDevice, G.st));
    gather_pad(G.tabA, G.batch, G.M, G.N, c.Ad, slab, G.st);
    if (gk) gather_pad(G.tabG, G.batch, G.N, G.M, c.Gd, slab, G.st);
    // alpha = 0: the recipe of a lone solve per instance (norms on the padded
    // slab are the instance's: zero padding adds zero rows and columns)
    for (int b = 0; b < G.batch; ++b) {
        if (alpha[b] == 0.0) {
            if (gk) {
                // P = GA or AG, chosen by the instance's own shape as a lone
                // solve does (padding can make the group's side differ when
                // the padded shape is square); one unbatched FP64 product into
                // the instance's s x s square, which fits either choice
                double* P = c.sq[0] + b * slab;
                const double* Ab = c.Ad + b * slab;
                const double* Gb = c.Gd + b * slab;
                const int keep = c.batch;
                c.batch = 1;
                if (G.d[b].m > G.d[b].n) gemm(c, G.N, G.N, G.M, Gb, G.M, false, Ab, G.N, false, epi1(term(P, c.s, 1)));
                else                     gemm(c, G.M, G.M, G.N, Ab, G.N, false, Gb, G.M, false, epi1(term(P, c.s, 1)));
                c.batch = keep;
                norms_1_inf(c.s, c.s, P, c.s, h->dsmall, c.red, G.st);
            } else {
                norms_1_inf(G.M, G.N, c.Ad + b * slab, G.N, h->dsmall, c.red, G.st);
            }
            CK(cudaMemcpyAsync(G.pinned, h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, G.st));
            CK(cudaStreamSynchronize(G.st));
            const double pr = G.pinned[0] * G.pinned[1];
            alpha[b] = (pr > 0 && std::isfinite(pr)) ? (gk ? 1.0 / std::sqrt(pr) : 1.0 / pr) : 1.0;
        }
        G.info[b].alpha = alpha[b];
        G.info[b].side = G.left ? 1 : 0;
    }
    CK(cudaMemcpyAsync(G.dalpha, alpha.data(), sizeof(double) * G.batch, cudaMemcpyHostToDevice, G.st));
    if (gk) scale_copy_batched(G.N, G.M, c.Gd, G.M, G.dalpha, c.X[0], G.M, slab, G.batch, G.st);
    else transpose_scale_batched(G.M, G.N, c.Ad, G.N, G.dalpha, c.X[0], G.M, slab, G.batch, G.st);
    // no wait here: the tables and alphas come from pageable host memory, which
    // cudaMemcpyAsync has consumed when it returns, and everything else is
    // ordered on the group's stream (a wait would hold the host -- and every
    // other group -- while this stream queues behind other work)
    CK(cudaPeekAtLastError());
    return PINV_OK;
}

// Issue loop k for every instance (asynchronous; norms land in pinned memory).
int group_issue_impl(Group& G) {
    Ctx& c = G.c;
    double maxrel = 0.0;   // the slowest running instance decides the group's class
    for (int b = 0; b < G.batch; ++b)
        if (!G.done[b]) maxrel = std::max(maxrel, G.prev_rel[b]);
    G.level = next_level(G.level, G.prev_prec, G.fp64_class, maxrel);
    c.prec_k = G.level;
    if (G.level == TC_BF16) G.bf16_ran = true;
    G.stab_now = G.stabilise && G.level == G.fp64_class;
    if (!G.serving) {
        // one-shot batches issue directly: a group runs ~9 loops, and capturing
        // and instantiating its graphs (~3 ms per group) costs more than the
        // launches it saves (measured 1354 vs 1214 ms for 4096 problems)
        const double* Xk = c.X[G.cur];
        double* Xn = c.X[G.cur ^ 1];
        int parts = pm_loop_f64(c, Xk, G.stab_now ? c.X[2] : Xn);
        if (G.stab_now) parts = stabilise_f64(c, c.X[2], Xk, Xn);
        if (parts < 0) return G.err = PINV_ERR_CUDA;
        G.parts = parts;
        reduce_pairs(c.partials, parts, G.dnorms, G.st, G.batch);
        CK(cudaMemcpyAsync(G.pinned, G.dnorms, sizeof(double) * 2 * G.batch, cudaMemcpyDeviceToHost, G.st));
        CK(cudaMemcpyAsync(G.pinned + 2 * G.batch, G.h->derr, sizeof(int), cudaMemcpyDeviceToHost, G.st));
        CK(cudaEventRecord(G.ev, G.st));
        G.in_flight = true;
        return PINV_OK;
    }
    // serving groups live for many loops next to other groups: their loop
    // chain is replayed as a CUDA graph (one per level, stabilised flag and
    // ping-pong side), which frees the host to feed the other groups
    const int key = (G.level * 2 + (G.stab_now ? 1 : 0)) * 2 + G.cur;
    auto it = G.graphs.find(key);
    if (it == G.graphs.end()) {
        // capture the loop: seven (or nine) products, the norm reduction and the
        // readback of the norms and the error word into pinned memory
        const int k0 = c.kernels;
        CK(cudaStreamBeginCapture(G.st, cudaStreamCaptureModeThreadLocal));
        const double* Xk = c.X[G.cur];
        double* Xn = c.X[G.cur ^ 1];
        int parts = pm_loop_f64(c, Xk, G.stab_now ? c.X[2] : Xn);
        if (G.stab_now) parts = stabilise_f64(c, c.X[2], Xk, Xn);
        if (parts >= 0) {
            reduce_pairs(c.partials, parts, G.dnorms, G.st, G.batch);
            cudaMemcpyAsync(G.pinned, G.dnorms, sizeof(double) * 2 * G.batch, cudaMemcpyDeviceToHost, G.st);
            cudaMemcpyAsync(G.pinned + 2 * G.batch, G.h->derr, sizeof(int), cudaMemcpyDeviceToHost, G.st);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(G.st, &graph);
        if (parts < 0 || ce != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            return G.err = PINV_ERR_CUDA;
        }
        // kernel nodes carry the group's stream priority explicitly, so replayed
        // loops of small problems keep overtaking the CTAs of large ones
        int prio = 0;
        if (cudaStreamGetPriority(G.st, &prio) == cudaSuccess && prio != 0) {
            size_t nn = 0;
            if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn) {
                std::vector<cudaGraphNode_t> nodes(nn);
                if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
                    for (cudaGraphNode_t node : nodes) {
                        cudaGraphNodeType type;
                        if (cudaGraphNodeGetType(node, &type) != cudaSuccess || type != cudaGraphNodeTypeKernel)
                            continue;
                        cudaLaunchAttributeValue v{};
                        v.priority = prio;
                        cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributePriority, &v);
                    }
            }
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return G.err = PINV_ERR_CUDA;
        it = G.graphs.emplace(key, exec).first;
        G.graph_parts[key] = parts;
        G.graph_kernels[key] = c.kernels - k0 + 1;
        c.kernels = k0;
    }
    CK(cudaGraphLaunch(it->second, G.st));
    c.kernels += G.graph_kernels[key];
    G.parts = G.graph_parts[key];
    CK(cudaEventRecord(G.ev, G.st));
    G.in_flight = true;
    return PINV_OK;
}

// Wait for loop k, apply the stop rule per instance, copy out stopped instances.
int group_complete_impl(Group& G) {
    CK(cudaEventSynchronize(G.ev));
    G.in_flight = false;
    int derr;
    std::memcpy(&derr, G.pinned + 2 * G.batch, sizeof(int));
    if (derr) return G.err = PINV_ERR_TIMEOUT;
    Ctx& c = G.c;
    const int k = G.k;
    const int prec_k = G.level;
    const bool final_class = prec_k == G.fp64_class && G.prev_prec == G.fp64_class;
    std::vector<int> mask(2 * G.batch, 0);
    bool any_copy = false, all_below_switch = true;
    for (int b = 0; b < G.batch; ++b) {
        if (G.done[b]) continue;
        pinv_info& I = G.info[b];
        const pinv_desc& x = G.d[b];
        const double dx2 = G.pinned[2 * b], x2 = G.pinned[2 * b + 1];
        const double e = stop_measure(&x, dx2, x2, k, I.alpha);
        I.loops_run = k + 1;
        if (k < PINV_HISTORY) { I.history[k] = e; I.precision[k] = (signed char)prec_k; }
        if (G.stab_now) ++I.stabilized_loops;
        const int maxit = x.max_iter ? x.max_iter : 100;
        int stop = 0;   // 1: keep X_k (buffer cur); 2: keep X_{k+1} (buffer cur^1)
        if (!std::isfinite(e)) { I.status = PINV_ERR_NONFINITE; stop = 1; }
        else if (e < x.tol && (x.stop != PINV_STOP_ORDER18 || prec_k == G.fp64_class)) {
            I.status = PINV_OK; I.stop_reason = 0; I.iters = k + 1; I.rel_step = e; stop = 2;
        }
        else {
            const double pv = G.prev[b];
            const bool stalled = G.stab_now ? (e >= pv) : (pv < 1e-3 && e >= pv * pv);
            const double rel = dx2 == 0.0 ? 0.0 : (x2 > 0 ? std::sqrt(dx2 / x2) : INFINITY);
            if (stalled && final_class) { I.status = PINV_OK; I.stop_reason = 1; I.iters = k; I.rel_step = pv; stop = 1; }
            else if (rel > 1e3 && k > 0) { I.status = PINV_ERR_DIVERGED; I.iters = k; stop = 1; }
            else if (k + 1 >= maxit) { I.status = PINV_ERR_MAXITER; I.stop_reason = 2; I.iters = k + 1; stop = 2; }
        }
        if (stop) {
            G.done[b] = 1;
            mask[stop == 1 ? b : G.batch + b] = 1;
            any_copy = true;
        } else {
            G.prev[b] = e;
            G.prev_rel[b] = dx2 == 0.0 ? 0.0 : (x2 > 0 ? std::sqrt(dx2 / x2) : INFINITY);
            I.rel_step = e;
            I.iters = k + 1;
            if (!(e < (x.switch_tol > 0 ? x.switch_tol : 1e-3))) all_below_switch = false;
        }
    }
    if (G.d[0].variant == PINV_VARIANT_STABILIZED && all_below_switch) G.stabilise = true;
    G.prev_prec = prec_k;
    if (any_copy) {
        // The host rewrites this mask only after the next loop's event, which the
        // stream orders after this copy, so no wait is needed.
        int* pm = G.loop_mask();
        std::memcpy(pm, mask.data(), sizeof(int) * 2 * G.batch);
        CK(cudaMemcpyAsync(G.dmask, pm, sizeof(int) * 2 * G.batch, cudaMemcpyHostToDevice, G.st));
        scatter_out(G.tabX, G.dmask, G.batch, G.N, G.M, c.X[G.cur], G.M, c.stride, G.st);
        scatter_out(G.tabX, G.dmask + G.batch, G.batch, G.N, G.M, c.X[G.cur ^ 1], G.M, c.stride, G.st);
    }
    G.cur ^= 1;
    G.k = k + 1;
    return PINV_OK;
}

// The finish step for every instance that ended with PINV_OK: restore its kept
// iterate, project, run one more loop, copy out.
// Issue the finish step of a group on its stream (no synchronisation; see
// group_finish).
int group_finish_issue_impl(Group& G) {
    if (!G.finish || G.err) return G.err;
    Ctx& c = G.c;
    std::vector<int> mask(G.batch, 0);
    bool any = false;
    for (int b = 0; b < G.batch; ++b)
        if (G.info[b].status == PINV_OK) { mask[b] = 1; any = true; }
    if (!any) return PINV_OK;
    int* pm = G.finish_mask();   // its own block: the last loop's mask copy may still be queued
    std::memcpy(pm, mask.data(), sizeof(int) * G.batch);
    CK(cudaMemcpyAsync(G.dmask, pm, sizeof(int) * G.batch, cudaMemcpyHostToDevice, G.st));
    scatter_in(G.tabX, G.dmask, G.batch, G.N, G.M, c.X[0], G.M, c.stride, G.st);
    c.prec_k = G.fp64_class;   // the finish runs in the schedule's final class
    pinv_desc d0 = G.d[0];
    cleanup_f64(c, &d0, c.X[0], c.X[1]);
    const int parts = !G.bf16_ran ? ns_step_f64(c, c.X[1], c.X[0]) : pm_loop_f64(c, c.X[1], c.X[0]);
    if (parts < 0) return G.err = PINV_ERR_CUDA;
    scatter_out(G.tabX, G.dmask, G.batch, G.N, G.M, c.X[0], G.M, c.stride, G.st);
    CK(cudaPeekAtLastError());
    return PINV_OK;
}

// The group steps record their first failure in G.err (a failing CUDA call
// returns its code through CK without touching the group), so callers that
// look only at G.err, like the serving rounds, see every error.
int group_record(Group& G, int r) {
    if (r && !G.err) G.err = r;
    return r;
}
int group_begin(Group& G) { return group_record(G, group_begin_impl(G)); }
int group_issue(Group& G) { return group_record(G, group_issue_impl(G)); }
int group_complete(Group& G) { return group_record(G, group_complete_impl(G)); }
int group_finish_issue(Group& G) { return group_record(G, group_finish_issue_impl(G)); }

int group_finish(Group& G) {
    if (group_finish_issue(G)) return G.err;
    if (G.finish) CK(cudaStreamSynchronize(G.st));
    return PINV_OK;
}

int pad_to(int x, int g) { return ((x + g - 1) / g) * g; }

// Run groups concurrently (one stream each): issue loop k of every active
// group, then complete them in order.
int run_groups(std::vector<std::unique_ptr<Group>>& groups) {
    int rc = PINV_OK;
    for (auto& g : groups) {
        int r = group_begin(*g);
        if (r) { g->err = r; rc = r; }
    }
    // Every group advances on its own: a group whose loop has finished on the
    // device is completed and issued its next loop (or, once its instances have
    // stopped, its finish) while the others are still computing, so small
    // groups do not wait for the largest group's loop at every step.
    std::vector<char> fin(groups.size(), 0);
    auto advance = [&](size_t i) {
        Group& g = *groups[i];
        if (!g.err && g.active() && g.k < g.max_iter) {
            if (group_issue(g)) rc = g.err;
        } else if (!fin[i]) {
            fin[i] = 1;
            if (int r = group_finish_issue(g)) { if (!g.err) g.err = r; rc = r; }
        }
    };
    for (size_t i = 0; i < groups.size(); ++i) advance(i);
    for (;;) {
        bool pending = false, progressed = false;
        for (size_t i = 0; i < groups.size(); ++i) {
            Group& g = *groups[i];
            if (g.err || !g.in_flight) continue;
            pending = true;
            if (cudaEventQuery(g.ev) == cudaErrorNotReady) continue;
            progressed = true;
            if (group_complete(g)) { rc = g.err; continue; }
            advance(i);
        }
        if (!pending) break;
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (size_t i = 0; i < groups.size(); ++i)
        if (!fin[i]) { fin[i] = 1; if (int r = group_finish_issue(*groups[i])) { if (!groups[i]->err) groups[i]->err = r; rc = r; } }
    for (auto& g : groups) {
        if (!g->err && g->finish && cudaStreamSynchronize(g->st) != cudaSuccess) rc = g->err = PINV_ERR_CUDA;
        for (auto& I : g->info) {
            if (g->err && I.status == PINV_OK) I.status = g->err;
            I.gemms = g->c.gemms;   // each instance's share of the group's executed work
            I.gemm_flops = g->c.gemm_flops / g->batch;
            I.tensor_flops = g->c.tensor_flops / g->batch;
        }
        g->release();
    }
    return rc;
}


// ------------------------------------------------------------------ serving
// Continuous batching at loop granularity: every pinv_poll runs one round.
//  1. admission: pending requests, oldest first, are bucketed by padded shape
//     and settings; each bucket becomes a new group if its memory fits under
//     the handle's HBM budget together with the groups already running
//     (otherwise admission stops: first come, first served);
//  2. every running group issues its next loop on its own stream, so groups
//     admitted in different rounds run on the device at the same time;
//  3. every group completes its loop (per-request stop rule); groups whose
//     requests have all stopped apply the finish step, report, free memory.
}  // namespace

struct pinv_handle::Running {
    std::unique_ptr<Group> g;
    std::vector<uint64_t> ids;
    size_t bytes = 0;
};

namespace {

int serve_round(pinv_handle* h) {
    using clock = std::chrono::steady_clock;
    // 1. admission
    std::map<std::vector<long long>, std::vector<uint64_t>> buckets;
    std::vector<std::vector<long long>> order;
    while (!h->queue.empty()) {
        const uint64_t id = h->queue.front();
        const pinv_desc& d = h->requests[id].desc;
        std::vector<long long> key = {pad_to(d.m, 64), pad_to(d.n, 64), d.kind, d.prec, d.variant, d.finish,
                                      d.stop};
        if (!buckets.count(key)) order.push_back(key);
        buckets[key].push_back(id);
        h->queue.pop_front();
    }
    std::deque<uint64_t> deferred;
    bool full = false;
    for (auto& key : order) {
        auto& ids = buckets[key];
        size_t o = 0;
        while (o < ids.size()) {
            const size_t n = std::min<size_t>(ids.size() - o, 256);
            const size_t bytes = group_bytes((int)n, (int)key[0], (int)key[1], (int)key[3],
                                             key[5] == PINV_FINISH_CLEAN, key[2] == PINV_OUTER_G);
            if (full || (h->budget && h->serving_bytes + bytes > h->budget)) {
                full = true;
                for (size_t j = o; j < ids.size(); ++j) deferred.push_back(ids[j]);
                break;
            }
            auto r = std::make_unique<pinv_handle::Running>();
            r->g = std::make_unique<Group>();
            r->g->h = h;
            r->g->serving = true;
            r->g->M = (int)key[0];
            r->g->N = (int)key[1];
            for (size_t j = o; j < o + n; ++j) {
                r->ids.push_back(ids[j]);
                r->g->d.push_back(h->requests[ids[j]].desc);
            }
            r->bytes = bytes;
            const int rc = group_begin(*r->g);
            h->n_admitted += r->ids.size();
            if (rc) {
                for (uint64_t id : r->ids) { h->requests[id].status = rc; h->requests[id].info.status = rc; }
                h->n_completed += r->ids.size();
                r->g->release();
            } else {
                h->n_running += (int)r->ids.size();
                h->serving_bytes += bytes;
                h->running.push_back(std::move(r));
            }
            o += n;
        }
    }
    for (auto it = deferred.rbegin(); it != deferred.rend(); ++it) h->queue.push_front(*it);
    // 2./3. every group advances on its own: a group whose loop has finished on
    // the device is completed and immediately issued its next loop; a group
    // still computing is left alone, so small problems are not held back by
    // large ones in other groups
    for (auto& r : h->running) {
        Group& G = *r->g;
        if (G.err) continue;
        if (G.in_flight) {
            if (cudaEventQuery(G.ev) != cudaSuccess) continue;
            group_complete(G);
        }
        if (!G.err && G.active() && G.k < G.max_iter) group_issue(G);
    }
    // retire finished groups
    for (size_t i = 0; i < h->running.size();) {
        auto& r = h->running[i];
        Group& G = *r->g;
        // a failed group retires at once (its memory is freed in stream order)
        if (!G.err && (G.in_flight || (G.active() && G.k < G.max_iter))) { ++i; continue; }
        group_finish(G);
        const auto now = clock::now();
        for (size_t j = 0; j < r->ids.size(); ++j) {
            auto& q = h->requests[r->ids[j]];
            q.info = G.info[j];
            if (G.err && q.info.status == PINV_OK) q.info.status = G.err;
            if (!G.done[j] && q.info.status == PINV_OK) q.info.status = PINV_ERR_MAXITER;
            q.info.ms = std::chrono::duration<float, std::milli>(now - q.t_submit).count();
            // the group's products ran for all its requests in lockstep: each
            // request's share of the executed work
            q.info.gemms = G.c.gemms;
            q.info.gemm_flops = G.c.gemm_flops / G.batch;
            q.info.tensor_flops = G.c.tensor_flops / G.batch;
            q.status = q.info.status;
        }
        G.release();
        h->serving_bytes -= r->bytes;
        h->n_completed += r->ids.size();
        h->n_running -= (int)r->ids.size();
        h->running.erase(h->running.begin() + i);
    }
    return PINV_OK;
}

}  // namespace

extern "C" {

int pinv_init(pinv_handle** out, const pinv_config* cfg) {
    if (!out) return PINV_ERR_ARG;
    *out = nullptr;
    pinv_handle* h = new pinv_handle();
    h->device = cfg ? cfg->device : 0;
    h->budget = cfg ? cfg->hbm_budget_bytes : 0;
    h->max_queued = cfg && cfg->max_queued > 0 ? cfg->max_queued : 0;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->dsmall, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->derr, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "pinv_init: %s\n", cudaGetErrorString(e));
        if (h->pinned) cudaFreeHost(h->pinned);
        delete h;
        return PINV_ERR_CUDA;
    }
    *out = h;
    return PINV_OK;
}

void pinv_destroy(pinv_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    h->running.clear();
    for (auto& g : h->loop_graphs) cudaGraphExecDestroy(g.exec);
    h->loop_graphs.clear();
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->dstate) cudaFree(h->dstate);
    if (h->hstate) cudaFreeHost(h->hstate);
    for (void* p : h->pinned_blocks) cudaFreeHost(p);
    h->pinned_blocks.clear();
    if (h->derr) cudaFree(h->derr);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    if (h->ws) cudaFree(h->ws);
    if (h->dsmall) cudaFree(h->dsmall);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
}

int pinv_solve(pinv_handle* h, const pinv_desc* desc, void* stream, pinv_info* info) {
    if (!h) return PINV_ERR_ARG;
    pinv_info local;
    pinv_info* out = info ? info : &local;
    if (cudaSetDevice(h->device) != cudaSuccess) return out->status = PINV_ERR_CUDA;
    return solve_one(h, desc, (cudaStream_t)stream, out);
}

int pinv_preconditioner(pinv_handle* h, const pinv_precond_desc* desc, void* stream, pinv_info* info) {
    if (!h) return PINV_ERR_ARG;
    pinv_info local;
    pinv_info* out = info ? info : &local;
    if (cudaSetDevice(h->device) != cudaSuccess) return out->status = PINV_ERR_CUDA;
    return precond_one(h, desc, (cudaStream_t)stream, out);
}

int pinv_solve_complex(pinv_handle* h, const pinv_desc* desc, void* stream, pinv_info* info) {
    if (!h) return PINV_ERR_ARG;
    pinv_info local;
    pinv_info* out = info ? info : &local;
    if (cudaSetDevice(h->device) != cudaSuccess) return out->status = PINV_ERR_CUDA;
    return solve_one(h, desc, (cudaStream_t)stream, out, true);
}

int pinv_solve_batched(pinv_handle* h, int count, const pinv_desc* descs, void* stream,
                       pinv_info* infos) {
    if (!h || count < 0 || (count && !descs)) return PINV_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return PINV_ERR_CUDA;
    for (int i = 0; i < count; ++i) {
        int rc = validate(&descs[i]);
        if (rc) return rc;
        if (descs[i].kind == PINV_DRAZIN || descs[i].kind == PINV_DRAZIN_NORMAL || descs[i].host_buffers ||
            descs[i].check || descs[i].prec == PINV_PREC_FP32_REFINE)
            return PINV_ERR_ARG;
    }
    // the caller's stream is ordered before the groups' streams
    cudaEvent_t ready;
    CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CK(cudaEventRecord(ready, (cudaStream_t)stream));
    CK(cudaEventSynchronize(ready));
    cudaEventDestroy(ready);
    // buckets: same settings and side, m and n padded to multiples of 64
    std::map<std::vector<long long>, std::vector<int>> buckets;
    for (int i = 0; i < count; ++i) {
        const pinv_desc& d = descs[i];
        const int Mp = pad_to(d.m, 64), Np = pad_to(d.n, 64);
        std::vector<long long> key = {Mp, Np, d.kind, d.prec, d.variant, d.finish, d.stop};
        buckets[key].push_back(i);
    }
    std::vector<std::unique_ptr<Group>> groups;
    std::vector<std::vector<int>> members;
    const int max_batch = 1024;
    for (auto& kv : buckets) {
        for (size_t o = 0; o < kv.second.size(); o += max_batch) {
            auto g = std::make_unique<Group>();
            g->h = h;
            g->M = (int)kv.first[0];
            g->N = (int)kv.first[1];
            std::vector<int> idx;
            for (size_t j = o; j < std::min(kv.second.size(), o + max_batch); ++j) {
                idx.push_back(kv.second[j]);
                g->d.push_back(descs[kv.second[j]]);
            }
            groups.push_back(std::move(g));
            members.push_back(idx);
        }
    }
    int rc = run_groups(groups);
    int worst = rc;
    for (size_t gi = 0; gi < groups.size(); ++gi)
        for (size_t j = 0; j < members[gi].size(); ++j) {
            const pinv_info& I = groups[gi]->info[j];
            if (infos) infos[members[gi][j]] = I;
            if (I.status != PINV_OK && worst == PINV_OK) worst = I.status;
        }
    return worst;
}

int pinv_submit(pinv_handle* h, const pinv_desc* desc, uint64_t* id) {
    if (!h || !desc || !id) return PINV_ERR_ARG;
    int rc = validate(desc);
    if (rc) return rc;
    if (desc->kind == PINV_DRAZIN || desc->kind == PINV_DRAZIN_NORMAL || desc->host_buffers || desc->check ||
        desc->prec == PINV_PREC_FP32_REFINE)
        return PINV_ERR_ARG;
    const size_t need = group_bytes(1, pad_to(desc->m, 64), pad_to(desc->n, 64), desc->prec,
                                    desc->finish == PINV_FINISH_CLEAN, desc->kind == PINV_OUTER_G);
    if (h->budget && need > h->budget) return PINV_ERR_BUDGET;
    std::lock_guard<std::mutex> lk(h->mu);
    if (h->max_queued && (int)h->queue.size() >= h->max_queued) {
        ++h->n_rejected;
        return PINV_ERR_BUSY;
    }
    ++h->n_submitted;
    *id = h->next_id++;
    pinv_handle::Request r;
    r.desc = *desc;
    r.t_submit = std::chrono::steady_clock::now();
    h->requests[*id] = r;
    h->queue.push_back(*id);
    return PINV_OK;
}

int pinv_poll(pinv_handle* h, uint64_t id, pinv_info* info) {
    if (!h) return PINV_ERR_ARG;
    std::lock_guard<std::mutex> lk(h->mu);
    auto it = h->requests.find(id);
    if (it == h->requests.end()) return PINV_ERR_UNKNOWN_ID;
    if (it->second.status == PINV_PENDING && (!h->queue.empty() || !h->running.empty())) {
        if (cudaSetDevice(h->device) != cudaSuccess) return PINV_ERR_CUDA;
        serve_round(h);
    }
    if (it->second.status == PINV_PENDING) return PINV_PENDING;
    const int st = it->second.status;
    if (info) *info = it->second.info;
    h->requests.erase(it);
    return st;
}

int pinv_serving_stats(pinv_handle* h, pinv_serving_counters* out) {
    if (!h || !out) return PINV_ERR_ARG;
    std::lock_guard<std::mutex> lk(h->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = h->n_submitted;
    out->rejected = h->n_rejected;
    out->admitted = h->n_admitted;
    out->completed = h->n_completed;
    out->queued = (int)h->queue.size();
    out->running = h->n_running;
    out->groups = (int)h->running.size();
    out->device_bytes = h->serving_bytes;
    return PINV_OK;
}

int pinv_alpha_estimate(pinv_handle* h, const pinv_desc* d, void* stream, double* alpha) {
    if (!h || !d || !alpha || !d->A || d->m < 1 || d->n < 1 || d->lda < d->n) return PINV_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return PINV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_workspace(h, std::max(h->ws_bytes, (size_t)(2 * 2 * 256 * sizeof(double))));
    if (rc) return rc;
    double* scratch = (double*)h->ws;
    norms_1_inf(d->m, d->n, d->A, d->lda, h->dsmall, scratch, st);
    CK(cudaMemcpyAsync(h->pinned, h->dsmall, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double p = h->pinned[0] * h->pinned[1];
    if (!(p > 0.0) || !std::isfinite(p)) return PINV_ERR_NONFINITE;
    *alpha = 1.0 / p;
    return PINV_OK;
}

int pinv_step(pinv_handle* h, int m, int n, const double* A, int lda, const double* X_in,
              double* X_out, int ldx, pinv_prec prec, int stabilized, void* stream,
              double* rel_step) {
    if (!h || m < 1 || n < 1 || !A || !X_in || !X_out || lda < n || ldx != m || X_in == X_out)
        return PINV_ERR_ARG;
    if (prec != PINV_PREC_FP64 && prec != PINV_PREC_MIXED_BF16 && prec != PINV_PREC_FP32 &&
        prec != PINV_PREC_FP64_TC && prec != PINV_PREC_BF16_FP32)
        return PINV_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return PINV_ERR_CUDA;
    pinv_desc d{};
    d.m = m; d.n = n; d.A = A; d.lda = lda; d.X = X_out; d.ldx = ldx;
    d.kind = PINV_MOORE_PENROSE; d.prec = prec;
    Ctx c{};
    cudaStream_t st = (cudaStream_t)stream;
    int rc = setup_context(h, &d, st, c);
    if (rc) return rc;
    c.prec_k = prec == PINV_PREC_FP64 ? 0 : (prec == PINV_PREC_MIXED_BF16 ? TC_BF16 :
               ((prec == PINV_PREC_FP32 || prec == PINV_PREC_BF16_FP32) ? TC_FP32 : TC_FP64));
    int parts = pm_loop_f64(c, X_in, stabilized ? c.X[2] : X_out);
    if (stabilized) parts = stabilise_f64(c, c.X[2], X_in, X_out);
    if (parts < 0) return PINV_ERR_CUDA;
    double dx2, x2;
    rc = read_norms(c, parts, &dx2, &x2);
    if (rc) return rc;
    if (rel_step) *rel_step = x2 > 0 ? std::sqrt(dx2 / x2) : INFINITY;
    CK(cudaGetLastError());
    return PINV_OK;
}

int pinv_drazin_index(pinv_handle* h, int n, const double* A, int lda, int max_index, void* stream, int* index,
                      int* ranks) {
    if (!h || n < 1 || !A || lda < n || max_index < 0 || max_index > 64 || !index) return PINV_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return PINV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    *index = -1;
    const size_t nn = (size_t)n * n;
    const size_t bytes = sizeof(double) * (3 * nn + 2 * 256);
    if (h->budget && bytes > h->budget) return PINV_ERR_BUDGET;
    double* buf = nullptr;
    CK(cudaMallocAsync((void**)&buf, bytes, st));
    double *P = buf, *Q = buf + nn, *X = buf + 2 * nn, *scratch = buf + 3 * nn;
    int rc = PINV_OK;
    if (cudaMemcpy2DAsync(P, sizeof(double) * n, A, sizeof(double) * lda, sizeof(double) * n, n,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        rc = PINV_ERR_CUDA;
    int prev = n;   // rank(A^0)
    if (ranks) ranks[0] = n;
    for (int k = 1; k <= max_index + 1 && rc == PINV_OK; ++k) {
        // rank(A^k) = trace(A^k (A^k)^dagger), the pseudoinverse by this library
        int r = 0;
        pinv_desc d{};
        d.m = d.n = n; d.A = P; d.lda = n; d.X = X; d.ldx = n;
        d.kind = PINV_MOORE_PENROSE;
        double alpha = 0.0;
        const int ra = pinv_alpha_estimate(h, &d, stream, &alpha);
        if (ra == PINV_ERR_NONFINITE) {
            r = 0;   // A^k = 0
        } else if (ra != PINV_OK) {
            rc = ra;
            break;
        } else {
            d.alpha = alpha;
            d.tol = 1e-12;
            d.stop = PINV_STOP_REL_FRO;
            d.prec = PINV_PREC_FP64_TC;
            d.variant = PINV_VARIANT_STABILIZED;
            d.finish = PINV_FINISH_CLEAN;
            pinv_info info;
            rc = solve_one(h, &d, st, &info);
            if (rc) break;
            trace_of_product(n, P, n, X, n, h->dsmall, scratch, st);
            if (cudaMemcpyAsync(h->pinned, h->dsmall, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = PINV_ERR_CUDA;
                break;
            }
            const double tr = h->pinned[0];
            if (!std::isfinite(tr)) { rc = PINV_ERR_NONFINITE; break; }
            r = (int)std::llround(tr);
        }
        if (ranks) ranks[k] = r;
        if (r == prev) { *index = k - 1; break; }
        prev = r;
        if (k <= max_index) {   // P <- P A
            rc = pinv_gemm(h, n, n, n, P, n, 0, A, lda, 0, Q, n, PINV_PREC_FP64_TC, stream);
            std::swap(P, Q);
        }
    }
    cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == PINV_OK) rc = PINV_ERR_CUDA;
    if (rc == PINV_OK && *index < 0) rc = PINV_ERR_MAXITER;
    return rc;
}

int pinv_autotune(pinv_handle* h, void* stream, int* crossover) {
    if (!h) return PINV_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return PINV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int sizes[] = {64, 128, 192, 256, 384, 512, 768, 1024};
    const int nmax = 1024;
    const TcMode mode = tc_mode(TC_FP64);
    const size_t mat = align_up(sizeof(double) * nmax * nmax);
    const size_t need = 3 * mat + align_up(tc_workspace_bytes(nmax, nmax, nmax, mode));
    int rc = ensure_workspace(h, std::max(need, h->ws_bytes));
    if (rc) return rc;
    double* A = (double*)h->ws;
    double* B = (double*)((char*)h->ws + mat);
    double* C = (double*)((char*)h->ws + 2 * mat);
    void* tcws = (char*)h->ws + 3 * mat;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int cross = 0;
    bool tc_won_all_above = true;
    for (int i = (int)(sizeof(sizes) / sizeof(sizes[0])) - 1; i >= 0; --i) {
        const int n = sizes[i];
        fill_pattern(n, n, A, n, 1u, st);
        fill_pattern(n, n, B, n, 2u, st);
        Epilogue e = epi1(term(C, n, 1));
        float ms[2] = {0, 0};
        for (int eng = 0; eng < 2; ++eng) {
            for (int rep = 0; rep < 4; ++rep) {   // first call warms up
                int kernels = 0;
                if (rep == 1) CK(cudaEventRecord(e0, st));
                if (eng == 0) gemm_f64(n, n, n, A, n, false, B, n, false, e, st, 1, 0, false,
                                       gemm_f64_pick_tile(n, n, 1, h->sms));
                else tc_gemm(n, n, n, A, n, false, B, n, false, e, mode, tcws, h->ws_bytes - 3 * mat, h->derr, st,
                             &kernels);
            }
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&ms[eng], e0, e1));
        }
        if (tc_won_all_above && ms[1] <= ms[0]) continue;   // tensor cores still faster here
        tc_won_all_above = false;
        cross = sizes[i] + 1;                                  // DMMA at this size and below
        break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    h->tc_crossover = cross;
    if (crossover) *crossover = cross;
    return PINV_OK;
}

int pinv_gemm(pinv_handle* h, int M, int N, int K, const double* A, int lda, int trans_a,
              const double* B, int ldb, int trans_b, double* C, int ldc, pinv_prec prec,
              void* stream) {
    if (!h || M < 1 || N < 1 || K < 1 || !A || !B || !C || ldc < N) return PINV_ERR_ARG;
    if (lda < (trans_a ? M : K) || ldb < (trans_b ? K : N)) return PINV_ERR_ARG;
    if (prec != PINV_PREC_FP64 && prec != PINV_PREC_MIXED_BF16 && prec != PINV_PREC_FP32 &&
        prec != PINV_PREC_FP64_TC && prec != PINV_PREC_BF16_FP32)
        return PINV_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return PINV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int pk = prec == PINV_PREC_FP64 ? 0 : (prec == PINV_PREC_MIXED_BF16 ? TC_BF16 :
                   ((prec == PINV_PREC_FP32 || prec == PINV_PREC_BF16_FP32) ? TC_FP32 : TC_FP64));
    Epilogue e = epi1(term(C, ldc, 1));
    if (pk == 0) {
        if (gemm_f64(M, N, K, A, lda, trans_a != 0, B, ldb, trans_b != 0, e, st, 1, 0, false,
                     gemm_f64_pick_tile(M, N, 1, h->sms)) < 0)
            return PINV_ERR_CUDA;
    } else {
        const size_t need = tc_workspace_bytes(M, N, K, tc_mode(pk));
        int rc = ensure_workspace(h, std::max(need, h->ws_bytes));
        if (rc) return rc;
        int kernels = 0;
        if (tc_gemm(M, N, K, A, lda, trans_a != 0, B, ldb, trans_b != 0, e, tc_mode(pk), h->ws, h->ws_bytes,
                    h->derr, st, &kernels, nullptr, nullptr, 1, 0, false, false, h->wait_limit) < 0)
            return PINV_ERR_CUDA;
    }
    CK(cudaMemcpyAsync(h->pinned + 2, h->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int derr;
    std::memcpy(&derr, h->pinned + 2, sizeof(int));
    if (derr) {
        cudaMemset(h->derr, 0, sizeof(int));
        return PINV_ERR_TIMEOUT;
    }
    CK(cudaGetLastError());
    return PINV_OK;
}

int pinv_set_wait_limit(pinv_handle* h, unsigned polls) {
    if (!h) return PINV_ERR_ARG;
    h->wait_limit = polls;
    return PINV_OK;
}

}  // extern "C"
