/*
 * pinv.h -- C ABI of the GB300 library for generalized inverses by the
 * order-18 hyperpower iteration of Pan, Soleymani and Zhao.
 *
 * The problem (Section 2): given A (m x n, real), an initial value
 * X0 = alpha * G with R(G) = T and N(G) = S, compute the outer inverse
 * X = A^(2)_{T,S}, the unique X with XAX = X, R(X) = T, N(X) = S (Section 1.1,
 * Eq. 1 and the lemma after it).  The Moore-Penrose inverse (G = A^T) and the
 * Drazin inverse (G = A^l, l >= ind(A)) are the special cases named in
 * Section 1.1; Section 4 gives their initial values.
 *
 * Each loop is the factorised seven-product step of Eq. PM (Section 2):
 *   R = I - AX,  R2 = R R,  R4 = R2 R2,
 *   M = (I + c1 R2 + R4)(I + c2 R2 + R4),
 *   T = M + c3 R2,  S = M + d1 R2 + d2 R4,
 *   X <- X (I + R)(T S + mu R2 + psi R4),
 * which equals X (I + R + ... + R^17) (Eq. hyper18).  The stabilised variant
 * appends X <- X A X (Eq. PM-modified, Section 7).  When n < m the library
 * forms the n x n residual I - XA and multiplies from the left; in exact
 * arithmetic this is the same iterate.
 *
 * Conventions for every entry point
 *   - Matrices are dense, real, row-major, with a leading dimension (elements
 *     between consecutive rows) >= the number of columns.
 *   - Unless a field says otherwise, matrix pointers are DEVICE pointers on the
 *     handle's device, owned by the caller; the library never frees them and
 *     reads/writes them only on the stream passed to the call.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.
 *   - Return value: PINV_OK or one of the PINV_ERR_* codes below.  On error the
 *     output matrix is unspecified and info->status (when info is given)
 *     repeats the code.
 *   - Device work never waits without a bound; no entry point traps or faults
 *     the GPU on bad input: arguments are validated on the host first.
 */
#ifndef PINV_H
#define PINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define PINV_OK              0
#define PINV_PENDING         1   /* pinv_poll: request not finished yet           */
#define PINV_ERR_ARG        -1   /* bad shape, leading dimension, kind, pointer   */
#define PINV_ERR_BUDGET     -2   /* workspace would exceed the HBM budget         */
#define PINV_ERR_NONFINITE  -3   /* NaN/Inf in a stop norm (bad input or blow-up) */
#define PINV_ERR_DIVERGED   -4   /* step size grew past the divergence guard      */
#define PINV_ERR_MAXITER    -5   /* max_iter loops without meeting a stop rule    */
#define PINV_ERR_TIMEOUT    -6   /* a bounded device-side wait gave up            */
#define PINV_ERR_CUDA       -7   /* a CUDA runtime call failed                    */
#define PINV_ERR_UNKNOWN_ID -8   /* pinv_poll: no such request                     */
#define PINV_ERR_BUSY       -9   /* pinv_submit: the admission queue is full (the
                                    request is rejected; nothing was queued)       */

/* ------------------------------------------------------------------ enums */
typedef enum {
    PINV_MOORE_PENROSE = 0,  /* G = A^T (Section 4; Theorem 6.2)                  */
    PINV_DRAZIN        = 1,  /* G = A^l, l = drazin_index >= ind(A) (Section 4)   */
    PINV_OUTER_G       = 2,  /* caller's G (n x m): A^(2)_{R(G),N(G)} (Thm 3.1), e.g.
                                the weighted Moore-Penrose inverse A^+_{MN}
                                (G = N^{-1} A^T M) or the Bott-Duffin inverse
                                (G = P_L) of Section 1.1                          */
    PINV_DRAZIN_NORMAL = 3   /* Drazin inverse from G = A^l (A^{2l+1})^T A^l: same
                                range and null space as A^D, GA has a real
                                nonnegative spectrum, so it converges whatever the
                                eigenvalues of A; alpha = 0 gives
                                1/sqrt(||GA||_1 ||GA||_inf)                          */
} pinv_kind;

typedef enum {
    PINV_STOP_REL_FRO = 0,   /* ||X_{k+1} - X_k||_F / ||X_k||_F < tol             */
    PINV_STOP_PAPER   = 1,   /* ||X_{k+1} - X_k||_F / (18^k alpha) < tol (Eq. stopreliable) */
    PINV_STOP_ORDER18 = 2    /* relative step < tol, with tol a threshold delta such
                                that delta^18 is below the unit roundoff of the final
                                product class (e.g. 1e-2 for FP64 class, 0.25 for
                                FP32 class):
                                by Theorem 3.1 (F_{k+1} = F_k^18) the loop that made
                                that step has reached the rounding floor; its result
                                is kept and no loop is spent observing the floor   */
} pinv_stop;

typedef enum {
    PINV_PREC_FP64       = 0, /* every product in native FP64 (DMMA)               */
    PINV_PREC_MIXED_BF16 = 1, /* loops in BF16 while the step is > 0.5 (growth phase),
                                 then FP32-class loops, then FP64-class (tensor cores)
                                 after the first FP32-class loop whose step is < 1.
                                 For problems without a null block (full column rank,
                                 nonsingular): on a rank-deficient problem BF16
                                 rounding lands in the null block, which grows by 18
                                 per loop (Theorem 6.2).  Needs alpha <= 1/sigma_max^2
                                 (e.g. the alpha = 0 recipe)                       */
    PINV_PREC_MIXED_FP8  = 2, /* reserved: FP8 early loops (returns PINV_ERR_ARG)  */
    PINV_PREC_FP32       = 3, /* FP32-class loops (4 exact BF16 slices, 10 slice
                                 products, 31 bits) while the iterate grows, then
                                 FP64-class loops after the first step below 1: the
                                 order-18 contraction of that loop removes the
                                 FP32-class rounding of the range.  Also for rank-
                                 deficient and rectangular problems (with the finish,
                                 which removes the rounding in the blocks the loop
                                 does not contract).  Needs alpha <= 1/sigma_max^2:
                                 with 2/(sigma_1^2 + sigma_r^2) the top residual
                                 eigenvalue sits at -1 and FP32-class rounding pushes
                                 it past                                         */
    PINV_PREC_FP64_TC    = 4, /* every product FP64-accurate on the BF16 tensor
                                 cores: 7 exact slices per operand, 28 products    */
    PINV_PREC_BF16_FP32  = 5, /* FP32-finished: BF16 while the step is > 0.5, then
                                 FP32-class to the end (the stop rule ends at the
                                 FP32 noise floor); the finish, if asked, in
                                 FP32-class products too.  Accuracy ~ u_fp32 *
                                 kappa; problems without a null block            */
    PINV_PREC_FP32_REFINE = 6 /* FP32-class loops of Eq. PM while the step is >= 1;
                                 the first loop whose step is below 1 is followed
                                 by X <- X A X in FP32 class (Section 7's stabilising
                                 product, counted in stabilized_loops), then order-2
                                 refinement steps X <- X + (I - XA) X (Eq. hyper,
                                 p = 2): the first in FP32 class, the others in
                                 FP64 class (R formed in FP64 class) until one's
                                 relative Frobenius change e_j, or the square of
                                 the previous step's e_{j-1} (each step squares
                                 the range error), is below 1e-5 (at most 16
                                 steps), then the finish; `stop` and
                                 `tol` are not used (the loops end at that switch,
                                 max_iter still bounds them).  Each refinement step squares the
                                 error of the range block, so two of them (4
                                 products, 2 of them FP64-class) replace the
                                 FP64-class order-18 loop (7 or 9 products) of
                                 PINV_PREC_FP32.  Single
                                 solves only (pinv_solve, pinv_solve_complex):
                                 the batched and served calls return PINV_ERR_ARG.
                                 Requires finish = PINV_FINISH_CLEAN and alpha <=
                                 1/sigma_max^2, as PINV_PREC_FP32, and kind
                                 PINV_MOORE_PENROSE or PINV_DRAZIN (the X A X
                                 finish of a general G leaves the FP32-class
                                 rounding: PINV_ERR_ARG).  The steps are
                                 recorded after the loops in info->history with
                                 precision codes 5 (FP32 class) and 6 (FP64) and
                                 counted in iters and loops_run                 */
} pinv_prec;

typedef enum {
    PINV_VARIANT_PLAIN      = 0, /* Eq. PM, 7 products per loop                    */
    PINV_VARIANT_STABILIZED = 1  /* Eq. PM-modified in the final-class loops after
                                    a step < switch_tol: 7 + 2 products per loop
                                    (the paper counts 8)                           */
} pinv_variant;

typedef enum {
    PINV_FINISH_NONE  = 0,
    PINV_FINISH_CLEAN = 1    /* after the loops: projection X <- (XA)^T X (AX)^T
                                (Moore-Penrose), A^l X^{2l+1} A^l (Drazin) or
                                X A X (general G: fixes any outer inverse),
                                then one order-2 step of the same family,
                                X <- X + (I - XA) X (Eq. hyper, p = 2), which
                                squares the projection's rounding (after BF16
                                loops: one order-18 loop instead); both in the
                                schedule's final class                          */
} pinv_finish;

/* --------------------------------------------------------------- structs */
typedef struct {
    size_t hbm_budget_bytes; /* cap on the handle's workspace; 0 = no cap           */
    int    device;           /* CUDA device ordinal                                 */
    int    max_queued;       /* serving: requests waiting for admission at most;
                                pinv_submit rejects further ones with
                                PINV_ERR_BUSY until admission drains the queue.
                                0 = no cap (the queue grows with the backlog)      */
    int    reserved[5];
} pinv_config;

/* Counters of the serving loop (pinv_serving_stats). */
typedef struct {
    uint64_t submitted;      /* pinv_submit calls that queued a request            */
    uint64_t rejected;       /* pinv_submit calls refused with PINV_ERR_BUSY      */
    uint64_t admitted;       /* requests moved from the queue into running groups  */
    uint64_t completed;      /* requests whose final status is known               */
    int      queued;         /* waiting for admission now (the backlog)            */
    int      running;        /* admitted and not yet completed                     */
    int      groups;         /* running groups (one stream each)                   */
    int      reserved;
    size_t   device_bytes;   /* device memory held by the running groups           */
} pinv_serving_counters;

typedef struct {
    int m, n;                /* A is m x n; X and G are n x m                       */
    const double *A; int lda;
    double       *X; int ldx;/* output; also the initial value when kind == OUTER_G
                                and G == NULL is not allowed                         */
    const double *G; int ldg;/* PINV_OUTER_G only                                    */
    pinv_kind    kind;
    int          drazin_index;  /* l >= ind(A), required for PINV_DRAZIN            */
    double       alpha;      /* > 0: X0 = alpha * G.  0: the Section 4 recipe:
                                1/(||A||_1 ||A||_inf) for MOORE_PENROSE,
                                1/Tr(A^{l+1}) for DRAZIN; for OUTER_G
                                1/sqrt(||P||_1 ||P||_inf), P = GA (m > n) or AG,
                                which bounds the spectral radius of GA and so
                                converges whenever GA has a real nonnegative
                                spectrum (weighted Moore-Penrose G = N^{-1}A^T M,
                                Bott-Duffin G = P_L with A positive definite,
                                G = I with A positive definite); one extra
                                product.  A = 0 (or GA = 0) takes alpha = 1:
                                X0 = 0 whatever alpha, and X = 0 is the answer    */
    double       tol;        /* stop tolerance for `stop`                            */
    pinv_stop    stop;
    int          max_iter;   /* 0 = the paper's 100 (Section 8)                      */
    pinv_prec    prec;
    pinv_variant variant;
    double       switch_tol; /* stabilised switch threshold; 0 = 1e-3                */
    pinv_finish  finish;     /* required (PINV_FINISH_CLEAN) for MIXED_BF16 / FP32
                                schedules when m != n: the block the iteration does
                                not contract keeps their rounding (PINV_ERR_ARG)   */
    int          host_buffers; /* 1: A, G and X are HOST pointers; the call copies
                                  A (and G) in and X out on `stream` and returns
                                  after the copy back has completed                  */
    int          check;      /* 1: fill info->penrose / info->drazin (extra GEMMs)   */
    int          profile;    /* 1: time every GEMM with CUDA events on `stream`
                                (info->gemm_ms / gemm_flops)                         */
    int          symmetric;  /* PINV_OUTER_G only: 1 asserts A is symmetric and G
                                commutes with it (e.g. G = I, the preconditioner
                                family), so the exact R is symmetric: the four
                                products of its even polynomial (R2, R4, M, TS)
                                compute half their tiles and mirror them.  R and
                                R Z stay full (their antisymmetric part corrects
                                the iterate).  Nonsingular A only.                 */
    int          reserved[2];
} pinv_desc;

/* Approximate-inverse preconditioner request (pinv_preconditioner). */
typedef struct {
    int n;                   /* A is n x n (square), X n x n                       */
    const double *A; int lda;
    double       *X; int ldx;/* output X_k                                          */
    int          loops;      /* loops of Eq. PM from X0, 1 .. PINV_HISTORY (the
                                paper's preconditioner is X_1)                     */
    double       alpha;      /* X0 = alpha diag(1/a_11 .. 1/a_nn); 0 = 1 (Eq. choice3) */
    double       chop;       /* > 0: after every loop, entries of magnitude < chop
                                become 0 (complex: real and imaginary parts
                                separately), the sparsification of Section 8,
                                Example 3 (it used 1e-5); 0: none                  */
    pinv_prec    prec;       /* product class: FP64 (DMMA), FP64_TC, FP32 (FP32-
                                class), MIXED_BF16 or BF16_FP32 (BF16 products)    */
    int          complex_matrix; /* 1: A and X are complex, interleaved (re, im)
                                    pairs, leading dimensions in complex elements  */
    int          host_buffers;   /* 1: A and X are host pointers (as in pinv_desc) */
    int          profile;        /* 1: time the GEMMs (info->gemm_ms)              */
    int          reserved[4];
} pinv_precond_desc;

#define PINV_HISTORY 128
typedef struct {
    int    status;           /* PINV_OK or the error code                           */
    int    iters;            /* loops whose result was kept                          */
    int    loops_run;        /* loops executed (one more when stopped at a minimum)  */
    int    stabilized_loops;
    int    stop_reason;      /* 0 tol met, 1 minimum, 2 max_iter                     */
    int    side;             /* 0: right residual I - AX (m x m); 1: left I - XA     */
    double rel_step;         /* stop measure of the last kept loop                   */
    double alpha;            /* alpha actually used                                  */
    double penrose[4];       /* relative ||AXA-A||, ||XAX-X||, ||AX-(AX)^T||, ||XA-(XA)^T|| */
    double drazin[3];        /* relative ||XAX-X||, ||AX-XA||, ||A^{l+1}X - A^l||     */
    float  ms;               /* wall time of the call on the host                    */
    int    gemms;            /* GEMM launches issued                                  */
    int    kernels;          /* all kernel launches issued (GEMMs included)          */
    float  gemm_ms;          /* desc->profile: summed CUDA-event time of the GEMMs   */
    double gemm_flops;       /* algorithmic flops of those GEMMs (2 M N K each)       */
    double tensor_flops;     /* BF16 tensor-core flops issued: 2 M N K per slice product */
    double history[PINV_HISTORY];  /* stop measure per loop                          */
    signed char precision[PINV_HISTORY]; /* per loop: 0 FP64, 1 BF16, 3 FP32-class,
                                            4 FP64-class; 5 / 6 an FP32- / FP64-
                                            class order-2 refinement step
                                            (PINV_PREC_FP32_REFINE)              */
} pinv_info;

typedef struct pinv_handle pinv_handle;

/* ---------------------------------------------------------- entry points */

/* Create a handle on cfg->device (cfg may be NULL: device 0, no budget).
 * The handle owns its workspace (grown on demand, kept between calls) and a
 * pinned host block for stop-norm readback.  PINV_ERR_CUDA if the device
 * cannot be used. */
int  pinv_init(pinv_handle **h, const pinv_config *cfg);

/* Release the handle and its workspace; never touches caller memory. */
void pinv_destroy(pinv_handle *h);

/* Solve one problem (Theorem 3.1 / Section 7): X0 from kind/alpha (Section 4),
 * then loops of Eq. PM (or Eq. PM-modified after the switch) until the stop
 * rule: the measure < tol; or, in the converged regime, a plain loop whose
 * step is not at least quadratically smaller than the previous one, or a
 * stabilised loop whose step did not decrease (the remark closing Section 6:
 * the iteration is not self-correcting; the iterate before that loop is
 * kept).  Blocks the host until the result is in desc->X.  Not re-entrant on
 * one handle. */
int  pinv_solve(pinv_handle *h, const pinv_desc *desc, void *stream, pinv_info *info);

/* Approximate-inverse preconditioner (Section 8, Example 3, and the closing
 * remark of the paper that one full loop of a high-order method already gives
 * one): X_k after desc->loops loops of Eq. PM (right residual I - AX) from the
 * Jacobi initial value X0 = alpha diag(1/a_ii) (Eq. choice3), each loop
 * followed by the chop when desc->chop > 0.  Without the chop,
 * I - X_k A = (I - X0 A)^(18^k): the preconditioned matrix X_k A is as close
 * to I as the 18^k-th power of the Jacobi iteration matrix allows.  There is
 * no stop rule: the loops run as asked.  info->history holds each loop's
 * relative step (before its chop), info->iters = loops.
 * PINV_ERR_ARG for a bad shape, a zero diagonal entry or an unknown prec;
 * PINV_ERR_NONFINITE if a step is not finite (X0 outside the convergence
 * region of Theorem 3.1 grows without bound). */
int  pinv_preconditioner(pinv_handle *h, const pinv_precond_desc *desc, void *stream, pinv_info *info);

/* Complex matrices (the paper's setting: A in C^{m x n}, A^* the conjugate
 * transpose, Section 1.1; Theorem 3.1 holds over C).  Same descriptor and
 * results as pinv_solve, with A, G and X complex: interleaved (re, im) double
 * pairs (the layout of C99 double _Complex and std::complex<double>), leading
 * dimensions counted in complex elements, X0 = alpha A^* for Moore-Penrose.
 * The library solves the real embedding E(Z) = [[Re Z, -Im Z], [Im Z, Re Z]]
 * (2m x 2n; E(ZW) = E(Z)E(W), E(Z^*) = E(Z)^T, so the iterates of E(A) are
 * the embeddings of the complex iterates) with every product formed as the
 * left column half of E(C) -- the four real products of a complex product --
 * and reads X off E(X).  Workspace: that of a real 2m x 2n solve.
 *   - alpha is real.  alpha = 0 takes 1/(||A||_1 ||A||_inf) with complex
 *     moduli (Moore-Penrose / general G) and 1/Re Tr(A^{l+1}) (Drazin: the
 *     paper's 1/Tr(A^{l+1}) is complex in general; its real part keeps
 *     |1 - alpha lambda^{l+1}| < 1 for the sector spectra the trace recipe
 *     needs).
 *   - Stop measures and residuals use complex Frobenius norms.
 *   - desc->symmetric must be 0 (PINV_ERR_ARG).  host_buffers works as in
 *     pinv_solve. */
int  pinv_solve_complex(pinv_handle *h, const pinv_desc *desc, void *stream, pinv_info *info);

/* Solve `count` independent Moore-Penrose or general-G problems (device
 * buffers).  Problems are grouped by shape padded to multiples of 64 and by
 * settings; each group runs the loop chain for all its problems in lockstep
 * (one launch per product for the whole group) on its own stream, groups
 * concurrently; each problem keeps its own alpha, stop rule and result.
 * Zero padding leaves every problem's iterate exact.  Blocks until done.
 * infos may be NULL or an array of `count`.  Returns PINV_OK or the first
 * non-OK problem status. */
int  pinv_solve_batched(pinv_handle *h, int count, const pinv_desc *descs, void *stream,
                        pinv_info *infos);

/* Non-blocking: queue a problem for the handle's serving loop and return its
 * id.  The descriptor is copied; A, G and X must stay valid until pinv_poll
 * reports a final status.  Moore-Penrose and general-G problems with device
 * buffers (PINV_ERR_ARG otherwise); PINV_ERR_BUDGET if the problem's device
 * memory alone exceeds the handle's HBM budget; PINV_ERR_BUSY (rejected, not
 * queued) when cfg->max_queued requests are already waiting for admission.
 * Thread-safe with pinv_poll.
 * Each group of requests runs on its own stream (by priority: smaller problems
 * first).  With the CUDA default of eight hardware queues, streams beyond
 * eight share queues and a small group's kernels can wait behind a large
 * group's; a serving process should set CUDA_DEVICE_MAX_CONNECTIONS=32 in its
 * environment before CUDA is initialised. */
int  pinv_submit(pinv_handle *h, const pinv_desc *desc, uint64_t *request_id);

/* Drive the serving loop one round and report request `id`.  A round admits
 * queued requests, oldest first, into groups of equal padded shape while their
 * memory fits under the HBM budget next to the groups already running; runs
 * one loop of every running group, each on its own stream, so requests that
 * arrived in different rounds compute at the same time; and retires groups
 * whose requests have all stopped.  Returns PINV_PENDING, or the request's
 * final status with *info filled (info->ms = submit-to-completion latency);
 * the request is then forgotten.  Results equal a lone pinv_solve of the same
 * request up to the rounding of the padded shape. */
int  pinv_poll(pinv_handle *h, uint64_t request_id, pinv_info *info);

/* Counters of the handle's serving loop: submitted, rejected (PINV_ERR_BUSY),
 * admitted and completed requests since pinv_init, and the current backlog
 * (queued), admitted requests still computing, their groups and the device
 * memory those hold.  Thread-safe with pinv_submit / pinv_poll.  No
 * counterpart in the paper (serving is this library's). */
int  pinv_serving_stats(pinv_handle *h, pinv_serving_counters *stats);

/* Section 4's scaling for rectangular A: *alpha = 1/(||A||_1 ||A||_inf),
 * computed on the device; desc->A (device) and shape are read. */
int  pinv_alpha_estimate(pinv_handle *h, const pinv_desc *desc, void *stream, double *alpha);

/* One loop from X_in to X_out (n x m device buffers, may not alias):
 * Eq. PM (stabilized = 0) or Eq. PM-modified (stabilized = 1), in `prec`
 * (FP64 or FP32-class or BF16 products), residual side chosen as in
 * pinv_solve.  *rel_step (host) receives ||X_out - X_in||_F / ||X_in||_F.
 * Exposed so one factorised loop can be checked against the naive order-18
 * step. */
int  pinv_step(pinv_handle *h, int m, int n, const double *A, int lda,
               const double *X_in, double *X_out, int ldx,
               pinv_prec prec, int stabilized, void *stream, double *rel_step);

/* C = op(A) op(B) (row-major, C is M x N) with the product engine of `prec`
 * (FP64: DMMA; FP64_TC/FP32/MIXED_BF16: the tcgen05 slice engine at FP64-,
 * FP32- or BF16-class accuracy), the building block of every loop above.
 * trans_a: A is stored K x M; trans_b: B is stored N x K.  Device pointers;
 * uses the handle's workspace. */
int  pinv_gemm(pinv_handle *h, int M, int N, int K, const double *A, int lda, int trans_a,
               const double *B, int ldb, int trans_b, double *C, int ldc, pinv_prec prec,
               void *stream);

/* The index of a square matrix, ind(A): the smallest l >= 0 with
 * rank(A^{l+1}) = rank(A^l) (the definition given with the Drazin initial
 * value in Section 4), for choosing drazin_index.  rank(A^k) is computed as
 * trace(A^k (A^k)^dagger) with this library's own Moore-Penrose solve
 * (FP64-class products, stabilised loops, finish), rounded to the nearest
 * integer; it counts the singular values the iteration resolves, so nonzero
 * singular values of A^k must stand well clear of rounding (above ~1e-8 of
 * the largest).  A (n x n, lda) is a device pointer; ranks (host, may be NULL)
 * receives rank(A^k) for k = 0 .. ind(A) + 1 and needs max_index + 2 entries.
 * *index = -1 and PINV_ERR_MAXITER when ind(A) > max_index (at most 64).
 * Device memory: three n x n matrices, stream-ordered, freed before return.
 * For a nonsingular A the index is 0; PINV_DRAZIN then needs drazin_index 1
 * (any l >= ind(A) gives A^D). */
int  pinv_drazin_index(pinv_handle *h, int n, const double *A, int lda, int max_index, void *stream,
                       int *index, int *ranks);

/* Autotune the product engine for FP64-class products on this device: time one
 * n x n x n product with the native FP64 (DMMA) kernel and with the tensor-core
 * slice engine for n = 64 ... 1024, and route FP64-class products whose largest
 * dimension is below the measured crossover to DMMA from then on (the tensor-
 * core engine's fixed costs -- slicing launches, 128 x 128 tiles -- dominate
 * small products).  *crossover (may be NULL) receives the size; 0 means the
 * tensor-core engine won everywhere.  The choice belongs to the handle. */
int  pinv_autotune(pinv_handle *h, void *stream, int *crossover);

/* Failure detection: the number of polls a device-side wait in the main loop
 * of the tensor-core product kernel makes before it gives up, for every later
 * call on this handle (0 restores the default, about a second of polling).
 * When a wait gives up the kernel records an error word, stops issuing work,
 * waits -- always with the default limit -- until the bulk copies and MMAs it
 * already issued have landed, releases its TMEM and returns; the call then
 * returns PINV_ERR_TIMEOUT and clears the word, so the next call starts clean.
 * A short limit makes such a wait run out on purpose (the operand copies take
 * longer than a few polls), which tests that path without a fault.  No
 * counterpart in the paper. */
int  pinv_set_wait_limit(pinv_handle *h, unsigned polls);

/* For callers that cannot allocate device memory (a plugin whose host
 * framework owns the allocator, code under a pool that forbids cudaMalloc,
 * code that must not trigger the implicit synchronisation of cudaMalloc or
 * cudaFree): the same FP64 loop as pinv_step, with every intermediate taken
 * from one fixed-size static device array inside the library, so the call
 * allocates nothing (no cudaMalloc/cudaFree/cudaMallocHost, no allocating
 * library routine).  The paper has no counterpart; this is a deployment aid.
 *   - No handle: runs on the current device; the caller passes A, X_in, X_out
 *     (device, n x m with ldx == m, X_in != X_out) and receives *rel_step.
 *   - m and n must be <= PINV_NOALLOC_MAX_DIM, else PINV_ERR_BUDGET with no
 *     device work.  The static array (about 1 MiB) lives on every GPU that
 *     loads the library until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls on a device share the array and it keeps the last call's
 *     contents: calls that overlap on the GPU race, so serialise them.
 *   - The call returns after `stream` has finished the loop: it synchronises
 *     the stream to read the two stop norms into *rel_step. */
#define PINV_NOALLOC_MAX_DIM 128
int  pinv_step_noalloc(int m, int n, const double *A, int lda, const double *X_in,
                       double *X_out, int ldx, int stabilized, void *stream,
                       double *rel_step);

#ifdef __cplusplus
}
#endif
#endif /* PINV_H */
