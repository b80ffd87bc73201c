// Tensor-core GEMM for every product of the iteration on sm_103a.
//
// C (M x N, FP64) = op(A) op(B) evaluated as a sum of BF16 slice products:
//   op(A) = sum_s A_s,  op(B) = sum_t B_t,   C = sum_{s + t <= L} A_s B_t.
// Slices are BF16 matrices.  In the exact modes (FP64-class, FP32-class) each
// row of op(A) (column of op(B)) is scaled by its power of two 2^-e (so its
// largest entry lies in [1/2, 1)), rounded to a T = 8S - 1 bit signed integer
// F and cut into S balanced base-256 digits: slice s holds q_s 2^(8(S-1-s) - T)
// with |q_s| <= 128, which bf16 (8 significant bits) holds exactly.  Every
// product q q' is an integer below 2^14 in magnitude times the power of two of
// its diagonal d = s + t, so every partial sum of a K-chunk of <= 1024 products
// is an integer multiple of that power of magnitude <= 2^24, which FP32 holds
// exactly -- the FP32 tensor-core accumulation is exact.  Each (pair, chunk)
// accumulator is drained from TMEM and summed exactly per diagonal in the
// epilogue, which combines the diagonals (exactly in int64 while the range
// allows, then in FP64) and finally applies 2^(e_i + f_j); the only rounding is
// the conversion to FP64 and the FP64 sum of the smallest diagonals, the
// rounding of F and the truncation of pairs with s + t > L.
//   FP64-class: 7 slices per operand (55 bits), s + t <= 6 (28 products)
//   FP32-class: 4 slices (31 bits), s + t <= 3 (10 products)
//   BF16:       1 slice rounded to nearest (no grid), one product
//
// Kernel layout (persistent, one CTA per SM walking the tiles, 10 warps; every
// CTA issues its own TMA loads):
//   warp 0      TMA producer: 3-D tensor maps [slice][row][k], 128B swizzle,
//               ragged edges zero-filled by the TMA unit
//   warp 1      TMEM allocator + single-thread tcgen05.mma issuer
//               (M = 128, N = BN, K = 16 per instruction, kind::f16, BF16 in,
//               FP32 accumulate), two TMEM accumulators so the epilogue drains
//               one while the next (pair, chunk) accumulates
//   warps 2..9  epilogue (two per TMEM lane quarter, 64 columns each): one
//               tcgen05.ld per drain, exact int32 sums per diagonal, int64
//               Horner / FP64 tile sums in TMEM, then the fused combination of
//               Eq. PM (identity, side inputs, up to three outputs) and the
//               stop-norm partials
// Every mbarrier wait is bounded; on timeout the kernel records an error code,
// waits (bounded) until its own bulk copies and MMAs in flight have landed,
// releases its TMEM and returns.

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "common.h"
#include "tc_gemm.h"

namespace pinv {
namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;          // 64 bf16 = one 128-byte swizzle row
constexpr int STAGES = 6;        // pipeline stages of products with several K-chunks
// Single-chunk products (short K: every tile is few units and the epilogue's
// fixed cost dominates) keep four stages: the shared memory given back becomes
// L1, which holds the epilogue's register spills and side inputs (4096-problem
// batch: 540 ms with six stages, 498 with four, 496 with three, 506 with five)
constexpr int LEAN_STAGES = 4;
constexpr int EPI_WARPS = 8;    // two per TMEM lane quarter, each owning BN/2 columns
constexpr int EPI_COLS = BN / 2;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int A_TILE_BYTES = BM * BK * 2;   // 16 KiB
constexpr int B_TILE_BYTES = BN * BK * 2;   // 16 KiB
constexpr int STAGE_BYTES = A_TILE_BYTES + B_TILE_BYTES;
// TMEM columns: two FP32 MMA accumulators [0, 2BN) and the FP64 running sums of
// the tile (two 32-bit columns per double) [2BN, 4BN).
constexpr int TMEM_COLS = 4 * BN;
constexpr unsigned WAIT_LIMIT = 1u << 22;   // polls before a wait gives up (about a second)

struct TcParams {
    int M, N, K;          // K = logical length (the tensor maps are zero-padded beyond it)
    int npairs;
    int pair_s[64], pair_t[64];
    // units of work: groups of consecutive pairs of one diagonal that share an
    // accumulator (more than one pair only when the whole K fits one chunk and
    // the group's products still sum exactly), times the K-chunks
    int ngroups;
    int grp_pair0[64], grp_npair[64];
    int chunk;            // K elements per exact accumulation
    int dint;             // diagonals 0..dint are summed exactly in int64 (Horner), -1: none
    int ubase;            // the Horner sums are in units of 2^-ubase (row-normalised)
    int hshift;           // the final fixed-point tile sums are in units of 2^-(ubase + hshift)
    int exact;            // 1: slices on power-of-two grids (integer-valued products)
    int S;                // slices per operand (tensor-map slice index = instance * S + s)
    int batch;            // instances; instance b uses every FP64 matrix at +b*stride
    long long stride;
    int sym;              // output symmetric (M == N): only tiles with nb >= mb, mirrored
    int tiles_m, tiles_n;
    Epilogue epi;
    // per output: which terms of out = a_acc acc + a_s1 s1 + a_s2 s2 + a_id I
    // are present, as integer flags (OUT_*), so that the final pass tests no
    // FP64 value: on GB300 every FP64 instruction -- a compare included -- holds
    // a sub-partition's FP64 unit for about 64 clocks per warp
    int okind[3];
    int* err;             // device error word (0 = ok)
    unsigned wait_limit;  // polls before a wait of the main loop gives up
    // bit patterns of the row maxima of op(A) and of the column maxima of op(B)
    // (exact modes): the epilogue scales each entry by 2^(e_i + f_j)
    const unsigned long long* rmax;
    const unsigned long long* cmax;
};

// Tile t of one instance -> (mb, nb).  Symmetric mode enumerates the upper
// triangle row by row: row mb holds tiles nb = mb .. tm-1.
__device__ __forceinline__ void tile_coords(int t, int tm, int sym, int& mb, int& nb) {
    if (!sym) { mb = t % tm; nb = t / tm; return; }
    mb = 0;
    while (t >= tm - mb) { t -= tm - mb; ++mb; }
    nb = mb + t;
}

// e with max = f 2^e, 1/2 <= f < 1 (0 for a zero maximum), by integer
// arithmetic on the bit pattern (GB300's FP64 pipe is narrow).
__device__ __forceinline__ int exponent_of(unsigned long long bits) {
    const int bexp = (int)((bits >> 52) & 0x7FF);
    if (bexp) return bexp - 1022;
    // zero or subnormal (m 2^-1074, 1 <= m < 2^52): 2^(p-1074) <= x < 2^(p-1073)
    const unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    return m ? (63 - __clzll((long long)m)) - 1073 : 0;
}
__device__ __forceinline__ int grid_exponent(const unsigned long long* mx, int i) { return exponent_of(mx[i]); }

// V 2^E for a 64-bit signed fixed-point value, rounded to nearest (ties to
// even), assembled from integer operations: GB300 issues about two FP64
// instructions per clock per SM, and the final pass of every tile would
// otherwise spend most of its time on the conversion and the scaling.  A
// result outside the normal range (subnormal, overflow; e.g. a NaN or infinity
// in a row maximum, whose exponent is huge) takes ldexp on the FP64 pipe.
// Out of line, so that the compiler cannot evaluate the FP64 conversion on
// every call and discard it (predication).
__device__ __noinline__ double fixed_to_double_slow(long long V, int E) { return ldexp((double)V, E); }
__device__ __noinline__ double float_to_double_slow(uint32_t f) { return (double)__uint_as_float(f); }
__device__ __noinline__ float double_to_float_slow(double x) { return __double2float_rn(x); }


// One path for every magnitude (normalise, keep 53 bits, round the 11 below
// them to nearest, ties to even): no divergence between the lanes of a warp.
__device__ __forceinline__ double fixed_to_double(long long V, int E) {
    const unsigned long long sign = (unsigned long long)V & 0x8000000000000000ull;
    const unsigned long long u = V < 0 ? 0ull - (unsigned long long)V : (unsigned long long)V;
    if (u == 0) return 0.0;
    const int lz = __clzll((long long)u);
    const unsigned long long n = u << lz;
    unsigned long long m = n >> 11;                       // 53-bit significand (may round up to 2^53)
    const unsigned rem = (unsigned)n & 0x7FFu;
    m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
    const int be = (63 - lz) + E + 1023;                  // biased exponent
    if (be < 1 || be > 2045) return fixed_to_double_slow(V, E);
    return __longlong_as_double((long long)(sign | (((unsigned long long)be << 52) + (m - (1ull << 52)))));
}

// The double of an FP32 bit pattern (exact), by integer operations for normal
// values.
__device__ __forceinline__ double float_bits_to_double(uint32_t f) {
    const uint32_t ex = (f >> 23) & 0xFFu;
    if ((f & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)((unsigned long long)f << 32));   // +-0
    if (ex == 0 || ex == 0xFFu) return float_to_double_slow(f);   // subnormal, inf, NaN
    const unsigned long long bits = ((unsigned long long)(f & 0x80000000u) << 32) |
                                    ((unsigned long long)(ex - 127 + 1023) << 52) |
                                    ((unsigned long long)(f & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// x rounded to FP32 (to nearest, ties to even) by integer operations on its
// bit pattern: the 29 fraction bits that FP32 lacks are dropped and the 23 it
// keeps rounded up when the dropped part is above half an FP32 unit, or
// exactly half with an odd last bit (a carry out of the fraction raises the
// exponent, and past the largest finite FP32 gives infinity, as IEEE 754
// rounding does).  Zeros stay exact; values that leave FP32's normal range
// (and infinities, NaNs) take the library conversion.
__device__ __forceinline__ float double_to_float(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    if (mag == 0) return __uint_as_float(sign);
    const int e = (int)(mag >> 52) - 1023 + 127;   // FP32 biased exponent
    if (e < 1 || e > 254) return double_to_float_slow(x);
    const uint32_t rem = (uint32_t)mag & 0x1FFFFFFFu;   // the 29 bits dropped
    uint32_t f = ((uint32_t)e << 23) | (uint32_t)((mag >> 29) & 0x7FFFFFu);
    f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(sign | f);
}


// 32-byte global accesses of four doubles (sm_100 and later); the address is
// 32-byte aligned
__device__ __forceinline__ void st_global_v4(double* p, double a, double b, double c, double d) {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(a), "d"(b), "d"(c), "d"(d) : "memory");
}
__device__ __forceinline__ void ld_global_v4(const double* p, double* v) {
    asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p)
                 : "memory");
}

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the phase with parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned limit = WAIT_LIMIT) {
    const uint32_t addr = smem_u32(bar);
    for (unsigned i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128B swizzle,
// 8-row core-matrix groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}
// Instruction descriptor, kind::f16: BF16 A/B, FP32 D, both K-major, M = 128, N = BN.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 columns of this warp's 32 TMEM lanes; the load and its wait are one asm
// statement, so no use of r[] can be scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld32_raw(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
// 16 columns (8 doubles of the tile sums) and the wait, in one asm statement.
__device__ __forceinline__ void tmem_ld16_raw(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
// 64 columns in one load (the whole drain of an epilogue warp), then the wait.
__device__ __forceinline__ void tmem_st32_raw(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void record_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ------------------------------------------------------------------ the kernel
// Final pass of one epilogue warp for one tile: its 32 rows (one per lane) x
// ncols columns of the tile sums in TMEM become
//   out = a_acc acc 2^(e_i + f_j) + a_s1 s1 + a_s2 s2 + a_id I
// for up to three outputs, plus the stop-norm partials of output 0 against s1,
// directly in the TMEM row layout.  On products with few units per tile this
// pass is most of the tile's latency, and on long products the next tile's
// MMAs wait on it; per element it does little: the column exponents of the
// tile are computed once per warp, the doubles are assembled with integer
// operations, each term is applied to a group's 8 values under one uniform
// test, the identity is tested only where the diagonal crosses, and each
// lane's row segment moves in 32-byte loads and stores.  (A variant staged
// through shared memory and stored in a column layout measured 0.5 % slower on
// the headline solve.)
__device__ __forceinline__ void final_pass(const TcParams& P, const Epilogue& E, uint32_t acc64, int row,
                                                int col0, int ncols, int row0w, const unsigned long long* rmax,
                                                const unsigned long long* cmax, int ew, bool mirror, int lane,
                                                double& sd, double& sx) {
    // the column exponents of this warp's half tile (static shared memory)
    __shared__ int ecol_all[EPI_WARPS][EPI_COLS];
    int* ecol = ecol_all[ew];
    if (rmax) {
        for (int cc = lane; cc < ncols; cc += 32) ecol[cc] = (col0 + cc < P.N) ? grid_exponent(cmax, col0 + cc) : 0;
        __syncwarp();
    }
    const bool rowok = row < P.M;
    const int erow = ((rmax && rowok) ? grid_exponent(rmax, row) : 0) - P.ubase - P.hshift;
    const double* s1 = (E.s1 && rowok) ? E.s1 + (size_t)row * E.ld1 : nullptr;
    const double* s2 = (E.s2 && rowok) ? E.s2 + (size_t)row * E.ld2 : nullptr;
    const bool norms = E.partials != nullptr;
#pragma unroll 1
    for (int c = 0; c < ncols; c += 8) {   // 8 columns per TMEM load
        uint32_t r[16];
        tmem_ld16_raw(acc64 + 2 * c, r);
        if (!rowok) continue;
        const int cb = col0 + c;                   // first column of the group
        const int ncol = min(8, P.N - cb);         // its valid columns
        if (ncol <= 0) continue;
        double a[8], v1[8];
        // the first side input's 8 values: two 32-byte loads when aligned and whole
        const bool v1wide = s1 && ncol == 8 && ((unsigned)reinterpret_cast<uintptr_t>(s1 + cb) & 31u) == 0;
        if (v1wide) {
            ld_global_v4(s1 + cb, v1);
            ld_global_v4(s1 + cb + 4, v1 + 4);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            // the tile sum in fixed point (exact modes)
            a[j] = fixed_to_double((long long)(((unsigned long long)r[2 * j + 1] << 32) | r[2 * j]),
                                   erow + (rmax ? ecol[c + j] : 0));
            if (!v1wide) v1[j] = (s1 && j < ncol) ? s1[cb + j] : 0.0;
        }
        const bool diag = cb < row0w + 32 && cb + 8 > row0w;   // the diagonal crosses this group
        const int dg = row - cb;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            if (o < E.nout) {
                const EpiTerm& t = E.o[o];
                const int kind = P.okind[o];
                double* out = (kind & OUT_STORE) ? t.out + (size_t)row * t.ld + cb : nullptr;
                const bool use_s2 = (kind & OUT_S2) && s2 != nullptr;
                // Each term of the combination is applied to the group's 8
                // values under one uniform test, its FP64 instructions inline
                // assembly: a term that is absent costs no FP64 instruction
                // (tested per element, the compiler evaluated every term and
                // selected -- about 4 FP64 instructions per element at ~64
                // clocks per warp each on GB300's FP64 pipe)
                double v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = (kind & OUT_NEG) ? neg(a[j]) : a[j];
                if (kind & OUT_MUL) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = dmul_keep(t.a_acc, v[j]);
                }
                if (kind & OUT_S1) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = dfma_keep(t.a_s1, v1[j], v[j]);
                }
                if (use_s2) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = dfma_keep(t.a_s2, j < ncol ? s2[cb + j] : 0.0, v[j]);
                }
                if ((kind & OUT_ID) && diag && dg >= 0 && dg < 8) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j == dg) v[j] = dadd_keep(v[j], t.a_id);
                }
                if (out) {
                    // a whole row segment leaves in two 32-byte stores when it is
                    // 32-byte aligned, else in four 16-byte ones when 16-byte aligned
                    const unsigned mis = (unsigned)reinterpret_cast<uintptr_t>(out) & 31u;
                    if (ncol == 8 && mis == 0) {
                        st_global_v4(out, v[0], v[1], v[2], v[3]);
                        st_global_v4(out + 4, v[4], v[5], v[6], v[7]);
                    } else if (ncol == 8 && (mis & 15u) == 0) {
#pragma unroll
                        for (int j = 0; j < 8; j += 2)
                            *reinterpret_cast<double2*>(out + j) = make_double2(v[j], v[j + 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j < ncol) out[j] = v[j];
                    }
                    if (mirror) {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j < ncol) t.out[(size_t)(cb + j) * t.ld + row] = v[j];   // warp-coalesced
                    }
                }
                if (o == 0 && norms) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (j < ncol) {
                            const double dd = dadd_keep(v[j], neg(v1[j]));
                            sd = dfma_keep(dd, dd, sd);
                            sx = dfma_keep(v1[j], v1[j], sx);
                        }
                    }
                }
            }
        }
    }
    if (rmax) __syncwarp();   // ecol is rewritten for the next tile
}


// Final pass of a BF16 product (one slice pair, FP32 accumulation): the same
// combination, outputs and stop-norm partials as final_pass, formed in FP32.
// The tile sum is already an FP32 value whose error is that of BF16 operands
// (relative 2^-8 and more); side inputs and coefficients are rounded to FP32
// (2^-24) and the FP32 result is stored exactly as a double.  No FP64
// instruction runs per element: the conversions are integer operations and
// the arithmetic is on the FP32 pipe, where GB300 issues about 64 times the
// FP64 rate.
__device__ __forceinline__ void final_pass_f32(const TcParams& P, const Epilogue& E, uint32_t acc64, int row,
                                               int col0, int ncols, int row0w, bool mirror, double& sd,
                                               double& sx) {
    const bool rowok = row < P.M;
    const double* s1 = (E.s1 && rowok) ? E.s1 + (size_t)row * E.ld1 : nullptr;
    const double* s2 = (E.s2 && rowok) ? E.s2 + (size_t)row * E.ld2 : nullptr;
    const bool norms = E.partials != nullptr;
    float fsd = 0.0f, fsx = 0.0f;
#pragma unroll 1
    for (int c = 0; c < ncols; c += 8) {   // 8 columns per TMEM load
        uint32_t r[16];
        tmem_ld16_raw(acc64 + 2 * c, r);
        if (!rowok) continue;
        const int cb = col0 + c;
        const int ncol = min(8, P.N - cb);
        if (ncol <= 0) continue;
        float v1[8];
        {
            double d1[8];
            if (s1 && ncol == 8 && ((unsigned)reinterpret_cast<uintptr_t>(s1 + cb) & 31u) == 0) {
                ld_global_v4(s1 + cb, d1);
                ld_global_v4(s1 + cb + 4, d1 + 4);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) d1[j] = (s1 && j < ncol) ? s1[cb + j] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) v1[j] = double_to_float(d1[j]);
        }
        const bool diag = cb < row0w + 32 && cb + 8 > row0w;
        const int dg = row - cb;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            if (o < E.nout) {
                const EpiTerm& t = E.o[o];
                const int kind = P.okind[o];
                double* out = (kind & OUT_STORE) ? t.out + (size_t)row * t.ld + cb : nullptr;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float a = __uint_as_float(r[2 * j]);
                    v[j] = (kind & OUT_NEG) ? -a : a;
                }
                if (kind & OUT_MUL) {
                    const float ca = double_to_float(t.a_acc);
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] *= ca;
                }
                if (kind & OUT_S1) {
                    const float c1 = double_to_float(t.a_s1);
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = fmaf(c1, v1[j], v[j]);
                }
                if ((kind & OUT_S2) && s2 != nullptr) {
                    const float c2 = double_to_float(t.a_s2);
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = fmaf(c2, double_to_float(j < ncol ? s2[cb + j] : 0.0), v[j]);
                }
                if ((kind & OUT_ID) && diag && dg >= 0 && dg < 8) {
                    const float ci = double_to_float(t.a_id);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j == dg) v[j] += ci;
                }
                if (out) {
                    double w[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) w[j] = float_bits_to_double(__float_as_uint(v[j]));
                    const unsigned mis = (unsigned)reinterpret_cast<uintptr_t>(out) & 31u;
                    if (ncol == 8 && mis == 0) {
                        st_global_v4(out, w[0], w[1], w[2], w[3]);
                        st_global_v4(out + 4, w[4], w[5], w[6], w[7]);
                    } else if (ncol == 8 && (mis & 15u) == 0) {
#pragma unroll
                        for (int j = 0; j < 8; j += 2)
                            *reinterpret_cast<double2*>(out + j) = make_double2(w[j], w[j + 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j < ncol) out[j] = w[j];
                    }
                    if (mirror) {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j < ncol) t.out[(size_t)(cb + j) * t.ld + row] = w[j];
                    }
                }
                if (o == 0 && norms) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (j < ncol) {
                            const float dd = v[j] - v1[j];
                            fsd = fmaf(dd, dd, fsd);
                            fsx = fmaf(v1[j], v1[j], fsx);
                        }
                    }
                }
            }
        }
    }
    sd = float_bits_to_double(__float_as_uint(fsd));
    sx = float_bits_to_double(__float_as_uint(fsx));
}

// LEAN: products of one K-chunk per pair (fewer stages); EXACT: the slice
// classes (fixed-point tile sums), else BF16 (FP32 accumulator, FP32 final
// pass), a separate instantiation so that the two final passes do not share
// one register allocation.
template <bool LEAN, bool EXACT>
__global__ void __launch_bounds__(THREADS, 1)   // 10 warps: 3 share a sub-partition (16K registers): <= 168 each
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               const __grid_constant__ TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int NST = LEAN ? LEAN_STAGES : STAGES;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STAGE_BYTES);
    uint64_t* empty = full + NST;
    uint64_t* accf = empty + NST;
    uint64_t* acce = accf + 2;
    uint64_t* drain = acce + 2;   // completion of every MMA the issuer launched
    uint64_t* tdone = drain + 1;  // every epilogue warp has finished with TMEM
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tdone + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_per = P.sym ? P.tiles_m * (P.tiles_m + 1) / 2 : P.tiles_m * P.tiles_n;
    const int ntiles = tiles_per * P.batch;
    const int work0 = (int)blockIdx.x;
    const int wstep = (int)gridDim.x;
    // tile w of the launch: instance b, blocks (mb, nb)
    auto locate = [&](int w, int& b, int& mb, int& nb) {
        b = w / tiles_per;
        tile_coords(w % tiles_per, P.tiles_m, P.sym, mb, nb);
    };
    const unsigned wl = P.wait_limit;
    const int kchunks = (P.K + P.chunk - 1) / P.chunk;
    const int units = P.ngroups * kchunks;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&accf[i], 1); mbar_init(&acce[i], 32 * EPI_WARPS); }
        mbar_init(drain, 1);
        mbar_init(tdone, EPI_WARPS);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_holder)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            // stages with a load issued (bit s), and the parity of its phase (bit s)
            uint32_t issued = 0, ipar = 0;
            for (int tile = work0; tile < ntiles && !*abort_flag; tile += wstep) {
                int b, mb, nb;
                locate(tile, b, mb, nb);
                const int m0 = mb * BM, n0 = nb * BN;
                for (int u = 0; u < units && !*abort_flag; ++u) {
                    const int grp = u / kchunks, ch = u % kchunks;
                    const int k_begin = ch * P.chunk;
                    const int k_end = min(P.K, k_begin + P.chunk);
                    for (int q = 0; q < P.grp_npair[grp] && !*abort_flag; ++q) {
                        const int pr = P.grp_pair0[grp] + q;
                        for (int k = k_begin; k < k_end; k += BK) {
                            if (!mbar_wait(&empty[stage], phase ^ 1, wl)) {
                                record_error(P.err, 1); *abort_flag = 1; break;
                            }
                            uint8_t* sa = smem + stage * STAGE_BYTES;
                            mbar_expect_tx(&full[stage], STAGE_BYTES);
                            tma_load_3d(sa, &mapA, &full[stage], k, m0, b * P.S + P.pair_s[pr]);
                            tma_load_3d(sa + A_TILE_BYTES, &mapB, &full[stage], k, n0, b * P.S + P.pair_t[pr]);
                            issued |= 1u << stage;
                            ipar = (ipar & ~(1u << stage)) | (phase << stage);
                            if (++stage == NST) { stage = 0; phase ^= 1; }
                        }
                    }
                }
            }
            // No bulk copy may still be writing into this CTA's shared memory when
            // it exits: wait (bounded, full limit) for the last load of every
            // stage.  A stage is reloaded only after its previous load was
            // consumed, so the last phase issued is the only one that can be
            // outstanding; on the normal path every wait returns at once.
            for (int s2 = 0; s2 < NST; ++s2)
                if ((issued >> s2) & 1u)
                    if (!mbar_wait(&full[s2], (ipar >> s2) & 1u)) record_error(P.err, 5);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            int stage = 0;
            uint32_t phase = 0;
            int buf = 0;
            uint32_t accphase[2] = {0, 0};
            for (int tile = work0; tile < ntiles && !*abort_flag; tile += wstep) {
                for (int u = 0; u < units && !*abort_flag; ++u) {
                    const int grp = u / kchunks, ch = u % kchunks;
                    const int k_begin = ch * P.chunk;
                    const int k_end = min(P.K, k_begin + P.chunk);
                    if (!mbar_wait(&acce[buf], accphase[buf] ^ 1, wl)) {
                        record_error(P.err, 2); *abort_flag = 1; break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + buf * BN;
                    uint32_t acc = 0;   // the group's pairs all add into one accumulator
                    for (int q = 0; q < P.grp_npair[grp] && !*abort_flag; ++q) {
                        for (int k = k_begin; k < k_end; k += BK) {
                            if (!mbar_wait(&full[stage], phase, wl)) {
                                record_error(P.err, 3); *abort_flag = 1; break;
                            }
                            tc_fence_after();
                            const uint32_t a0 = smem_u32(smem + stage * STAGE_BYTES);
                            const uint32_t b0 = a0 + A_TILE_BYTES;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                mma_bf16(d, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc, acc);
                                acc = 1;
                            }
                            mma_commit(&empty[stage]);
                            if (++stage == NST) { stage = 0; phase ^= 1; }
                        }
                    }
                    mma_commit(&accf[buf]);
                    accphase[buf] ^= 1;
                    buf ^= 1;
                }
            }
            // every MMA this thread issued has finished (reading shared memory,
            // writing TMEM) before the CTA releases either: on the normal path the
            // epilogue has already drained them all
            mma_commit(drain);
            if (!mbar_wait(drain, 0)) record_error(P.err, 6);
        }
    } else {
        // ---------------------------------------------------------- epilogue (warps 2..9)
        // Drained accumulators of one slice diagonal d = s + t share the unit
        // 2^-(14+8d) (the slices are integer digits times powers of two), so in
        // the exact modes they are summed exactly as int32: each drain is at
        // most 2^24 units, and at most 127 drains are summed before the int32
        // sums are added to the running sums of the tile in TMEM columns
        // [2BN, 4BN) (once per diagonal, or every 127 drains).  Diagonals 0..dint go into
        // an exact int64 by Horner's rule (C <- 256 C + I_d on the integer
        // pipe; the host picks dint so that |C| < 2^62).  The later diagonals
        // (2^-8(d-dint) of the unit and smaller) are summed in FP32 registers,
        // whose rounding lies far below the truncation of the slice pairs, and
        // after the last unit the tile sum becomes one fixed-point integer
        // V = C 2^h + round(F 2^h) (units 2^-(ubase+h), |V| < 2^62).  The final
        // pass turns V into a double with integer operations; FP64
        // instructions -- about 2 per clock per SM on GB300 -- are left to the
        // fused combination only.  BF16 products (one unit) keep the FP32
        // accumulator bits, and their final pass forms the combination in FP32.
        const int lg = warp & 3;                 // TMEM lane group of this warp
        const int half = (warp - 2) >> 2;        // which BN/2 columns of the tile
        const int ew = warp - 2;                 // epilogue warp index
        const uint32_t lane_base = tmem + ((uint32_t)(lg * 32) << 16);
        const uint32_t acc64 = lane_base + 2 * BN + 2 * half * EPI_COLS;   // this warp's tile sums
        int buf = 0;
        uint32_t accphase[2] = {0, 0};
        for (int tile = work0; tile < ntiles; tile += wstep) {
            int b, mb, nb;
            locate(tile, b, mb, nb);
            const int m0 = mb * BM, n0 = nb * BN;
            // A tile with at most BN/2 valid columns (a narrow single-chunk
            // product, or the last tile column of one) is split between both
            // warps of a lane quarter, BN/4 valid columns each, instead of
            // leaving one of them idle: each warp drains its 32 valid columns
            // as its first 32 (and 32 columns past N as the rest), so the final
            // pass -- most of such a tile's latency -- covers half the columns.
            const bool narrow = LEAN && P.N - n0 <= EPI_COLS;
            const int ncols = narrow ? EPI_COLS / 2 : EPI_COLS;   // valid columns of this warp
            const int cbase = half * ncols;                          // the first of them
            // slot of the tile's partials (instance-major, nb-major then mb)
            const int slot = b * P.tiles_m * P.tiles_n + nb * P.tiles_m + mb;
            const bool mirror = P.sym && mb != nb;   // also write the transposed tile
            const long long off = (long long)b * P.stride;   // instance b's matrices
            Epilogue E = P.epi;   // instance b's matrices, held in registers
            if (E.s1) E.s1 += off;
            if (E.s2) E.s2 += off;
            for (int o = 0; o < 3; ++o)
                if (E.o[o].out) E.o[o].out += off;
            const unsigned long long* rmax = P.rmax ? P.rmax + (size_t)b * P.M : nullptr;
            const unsigned long long* cmax = P.cmax ? P.cmax + (size_t)b * P.N : nullptr;
            int iacc[EPI_COLS];
            int ndrain = 0;   // drains summed in iacc since its last flush
            int hdiag = -1;   // diagonal of the last flush
            bool have64 = false;
            bool ok = true;
            for (int u = 0; u < units; ++u) {
                const int pr = P.grp_pair0[u / kchunks];   // every pair of the group has this diagonal
                const int d = P.pair_s[pr] + P.pair_t[pr];
                if (ndrain == 0) {
#pragma unroll
                    for (int j = 0; j < EPI_COLS; ++j) iacc[j] = 0;
                }
                if (*abort_flag || !mbar_wait(&accf[buf], accphase[buf], wl)) {
                    record_error(P.err, 4); *abort_flag = 1; ok = false; break;
                }
                tc_fence_after();
                const uint32_t taddr = lane_base + buf * BN + cbase;   // first 32 columns
                const uint32_t taddr2 = narrow ? lane_base + buf * BN + EPI_COLS + cbase : taddr + 32;
                const int uexp = 14 + 8 * d;   // slice products q q' 2^-(14+8d): accumulator / unit
                const bool horner = EXACT && d <= P.dint;
                // exact diagonals: the accumulator in integer units; later ones:
                // FP32 in units of 2^-ubase
                const float unit = ldexpf(1.0f, horner ? uexp : P.ubase);
#pragma unroll
                for (int hh = 0; hh < EPI_COLS; hh += 32) {
                    // the drain in two 32-column loads, each converted at once (32
                    // registers in flight next to the 64 of the sums, not 64); the
                    // accumulator goes back to the MMA issuer after the second load
                    uint32_t r[32];
                    tmem_ld32_raw(hh ? taddr2 : taddr, r);
                    if (hh + 32 == EPI_COLS) {
                        tc_fence_before();
                        mbar_arrive(&acce[buf]);
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        if (horner) iacc[hh + j] += __float2int_rn(__uint_as_float(r[j]) * unit);
                        else if (EXACT)
                            iacc[hh + j] = __float_as_int(fmaf(__uint_as_float(r[j]), unit, __int_as_float(iacc[hh + j])));
                        else iacc[hh + j] = (int)r[j];   // one drain only: keep the FP32 bits
                    }
                }
                accphase[buf] ^= 1;
                buf ^= 1;
                const bool last = u + 1 == units;
                const bool diag_done =
                    last || (P.pair_s[P.grp_pair0[(u + 1) / kchunks]] + P.pair_t[P.grp_pair0[(u + 1) / kchunks]] != d);
                const long long hmul = 1LL << P.hshift;
                if (horner) {
                    if (diag_done || ++ndrain == 127) {   // add the int32 sums to the Horner sums in TMEM
                        ndrain = 0;
                        const bool shift = have64 && d != hdiag;   // first flush of diagonal d > 0
#pragma unroll
                        for (int c = 0; c < EPI_COLS; c += 16) {
                            uint32_t r[32];
                            if (have64) tmem_ld32_raw(acc64 + 2 * c, r);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                long long C = have64 ? (long long)(((unsigned long long)r[2 * j + 1] << 32) | r[2 * j])
                                                     : 0LL;
                                if (shift) C *= 256;
                                C += iacc[c + j];
                                if (last) C *= hmul;   // every diagonal was exact: the final fixed point
                                r[2 * j] = (uint32_t)(unsigned long long)C;
                                r[2 * j + 1] = (uint32_t)((unsigned long long)C >> 32);
                            }
                            tmem_st32_raw(acc64 + 2 * c, r);
                        }
                        have64 = true;
                        hdiag = d;
                    }
                } else {
                    ndrain = 1;   // FP32 sums run on to the last unit without a flush
                    if (last) {   // V = C 2^h + round(F 2^h), or the FP32 bits of a BF16 product
                        const float fh = ldexpf(1.0f, P.hshift);
#pragma unroll
                        for (int c = 0; c < EPI_COLS; c += 16) {
                            uint32_t r[32];
                            if (have64) tmem_ld32_raw(acc64 + 2 * c, r);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                if (EXACT) {
                                    long long V = have64 ? (long long)(((unsigned long long)r[2 * j + 1] << 32) | r[2 * j])
                                                         : 0LL;
                                    V = V * hmul + __float2ll_rn(__int_as_float(iacc[c + j]) * fh);
                                    r[2 * j] = (uint32_t)(unsigned long long)V;
                                    r[2 * j + 1] = (uint32_t)((unsigned long long)V >> 32);
                                } else {
                                    r[2 * j] = (uint32_t)iacc[c + j];
                                    r[2 * j + 1] = 0u;
                                }
                            }
                            tmem_st32_raw(acc64 + 2 * c, r);
                        }
                        have64 = true;
                    }
                }
            }
            if (!ok) break;
            double sd = 0.0, sx = 0.0;
            if (EXACT)
                final_pass(P, E, acc64, m0 + lg * 32 + lane, n0 + cbase, ncols, m0 + lg * 32, rmax, cmax, ew,
                           mirror, lane, sd, sx);
            else
                final_pass_f32(P, E, acc64, m0 + lg * 32 + lane, n0 + cbase, ncols, m0 + lg * 32, mirror, sd, sx);
            if (P.epi.partials) {  // one pair per (tile, epilogue warp): no barrier between warps
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    sd += __shfl_xor_sync(0xffffffffu, sd, off);
                    sx += __shfl_xor_sync(0xffffffffu, sx, off);
                }
                if (lane == 0) {
                    P.epi.partials[2 * (EPI_WARPS * slot + ew)] = sd;
                    P.epi.partials[2 * (EPI_WARPS * slot + ew) + 1] = sx;
                }
            }
        }
        // this warp is done with TMEM (normal end or abort): tell the deallocator
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tdone);
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // The CTA barrier above is not relied on to order the epilogue warps'
        // last TMEM loads before the release (measured: the producer and MMA
        // warps can leave it while the epilogue warps are still in their final
        // pass); the release waits for every epilogue warp's arrival instead.
        if (lane == 0 && !mbar_wait(tdone, 0)) record_error(P.err, 7);
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// ------------------------------------------------------------------ slicing
// One operand's row maxima pass: rows of op(X) (op(X)[i][k] = trans ? X[k][i]
// : X[i][k]); mx[i] receives the bit pattern of max_k |op(X)[i][k]|
// (non-negative doubles order like their bits, so integer max is the floating
// max, taken on the integer pipe; a NaN or infinity wins and poisons the row).
// gx x gy blocks of 256 threads per instance: one row per warp (trans = 0), or
// a (32 columns) x (256 rows of X) patch per block, coalesced along the
// columns and combined with atomicMax into a zeroed mx (trans = 1).
struct MaxOp {
    int rows, K;
    const double* X;
    int ld, trans;
    unsigned long long* mx;
    long long stride;
    int gx, gy;
};
__device__ __forceinline__ void absmax_block(const MaxOp& o, int bx, int by, int bz, unsigned long long (*sh)[33]) {
    const double* X = o.X + (long long)bz * o.stride;
    unsigned long long* mx = o.mx + (size_t)bz * o.rows;
    const unsigned long long* Xb = reinterpret_cast<const unsigned long long*>(X);
    constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (!o.trans) {
        const int i = bx * 8 + w;
        if (i >= o.rows) return;
        unsigned long long m = 0;
        for (int k = lane; k < o.K; k += 32) m = max(m, Xb[(size_t)i * o.ld + k] & ABS);
        for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) mx[i] = m;
        return;
    }
    const int i = bx * 32 + lane;
    const int k0 = by * 256, k1 = min(o.K, k0 + 256);
    unsigned long long m = 0;
    if (i < o.rows)
        for (int k = k0 + w; k < k1; k += 8) m = max(m, Xb[(size_t)k * o.ld + i] & ABS);
    sh[w][lane] = m;
    __syncthreads();
    if (w == 0 && i < o.rows) {
        for (int j = 1; j < 8; ++j) m = max(m, sh[j][lane]);
        atomicMax(&mx[i], m);
    }
}
// The maxima passes of both operands of a product in one launch: blocks
// [0, a.gx a.gy) serve a, the rest b; blockIdx.y is the instance.
__global__ void __launch_bounds__(256) absmax_pair_kernel(MaxOp a, MaxOp b) {
    __shared__ unsigned long long sh[8][33];
    const int na = a.gx * a.gy;
    const int id = (int)blockIdx.x;
    if (id < na) absmax_block(a, id % a.gx, id / a.gx, blockIdx.y, sh);
    else absmax_block(b, (id - na) % b.gx, (id - na) / b.gx, blockIdx.y, sh);
}

// out[s][i][k] (bf16, row length Kp, Kp a multiple of 8) for 32 x 64 tiles of
// op(X); zero beyond K.  Each of the 256 threads turns 8 consecutive k of one
// row into one 16-byte store per slice plane.  exact = 1: base-256 digit
// slices of the row-normalised value (slice s holds q_s 2^(8(S-1-s) - T),
// T = 8S - 1); exact = 0: one round-to-nearest slice.
struct SliceOp {
    int rows, K, Kp;
    const double* X;
    int ld, trans;
    const unsigned long long* mx;
    int S, exact;
    __nv_bfloat16* out;
    long long stride;
    int gx, gy;   // (Kp / 64) x (rows / 32) tiles per instance
};
__device__ __forceinline__ void slice_tile(const SliceOp& o, int bx, int by, int bz, double (*t)[33]) {
    const int rows = o.rows, K = o.K, Kp = o.Kp, ld = o.ld, trans = o.trans, S = o.S, exact = o.exact;
    const double* X = o.X + (long long)bz * o.stride;   // instance bz
    __nv_bfloat16* out = o.out + (size_t)bz * S * rows * Kp;
    const unsigned long long* mx = o.mx ? o.mx + (size_t)bz * rows : nullptr;
    const int i0 = by * 32, k0 = bx * 64;
    const int tid = threadIdx.x;
    const int il = tid >> 3, kb = k0 + (tid & 7) * 8;   // row in the tile, first of 8 k
    const int i = i0 + il;
    double v[8];
    if (trans) {   // X is K x rows: coalesced along i into shared memory, then 8 k per thread
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int kr = (tid >> 5) + 8 * r, ic = tid & 31;
            const int k = k0 + kr, ii = i0 + ic;
            t[kr][ic] = (k < K && ii < rows) ? X[(size_t)k * ld + ii] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = t[(tid & 7) * 8 + j][il];
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (i < rows && kb + j < K) ? X[(size_t)i * ld + kb + j] : 0.0;
    }
    if (i >= rows || kb >= Kp) return;
    const size_t plane = (size_t)rows * Kp;
    uint4* dst = reinterpret_cast<uint4*>(out + (size_t)i * Kp + kb);   // 16-byte aligned: Kp, kb multiples of 8
    const size_t pstep = plane / 8;                                       // planes apart, in uint4
    auto pack = [](__nv_bfloat16 a, __nv_bfloat16 b) {
        return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
    };
    if (!exact) {   // one slice, FP64 rounded to nearest bf16 directly
        uint4 w;
        w.x = pack(__double2bfloat16(v[0]), __double2bfloat16(v[1]));
        w.y = pack(__double2bfloat16(v[2]), __double2bfloat16(v[3]));
        w.z = pack(__double2bfloat16(v[4]), __double2bfloat16(v[5]));
        w.w = pack(__double2bfloat16(v[6]), __double2bfloat16(v[7]));
        dst[0] = w;
        const uint4 zero = make_uint4(0, 0, 0, 0);
        for (int s = 1; s < S; ++s) dst[s * pstep] = zero;
        return;
    }
    // 2^ei > max |row i| (max = f 2^ei, 1/2 <= f < 1)
    const int ei = exponent_of(mx[i]);
    const int T = 8 * S - 1;
    // Integer digit extraction (GB300's FP64 pipe is narrow): x = m 2^E with a
    // 53-bit integer m; U = round(|x| / 2^(ei - T)) <= 2^T is a fixed-point
    // integer; its balanced base-256 digits (the lower ones in [-128, 127], the
    // top one <= 128 because U <= 2^T) are read off W = U + 128 (1 + 256 + ...
    // + 256^(S-2)): digit b (from the bottom) = byte b of W - 128, the top one
    // W >> 8(S-1) -- the carries of the digit-by-digit rule (byte + carry >=
    // 128: digit - 256, carry 1) happen in the one addition.  Then q_s =
    // +-digit, |q_s| <= 128.  A NaN or infinity poisons every slice so that
    // the product reports it.
    uint32_t lo[8], hi[8];
    int sgn[8];
    bool bad[8];
    unsigned long long bias = 0;
    for (int b = 0; b < S - 1; ++b) bias |= 0x80ull << (8 * b);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long bits = __double_as_longlong(v[j]);
        const int bexp = (int)((bits >> 52) & 0x7FF);
        bad[j] = bexp == 0x7FF;
        const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (bexp ? (1LL << 52) : 0LL);
        const int E = (bexp ? bexp : 1) - 1075;         // x = mant * 2^E
        const int shift = E - (ei - T);                 // U = mant * 2^shift
        unsigned long long U;
        if (shift >= 0) U = (unsigned long long)mant << shift;   // <= 2^T <= 2^55 since |x| < 2^ei
        else if (shift > -62) U = (unsigned long long)((mant + (1LL << (-shift - 1))) >> (-shift));
        else U = 0;
        U += bias;
        lo[j] = (uint32_t)U;
        hi[j] = (uint32_t)(U >> 32);
        sgn[j] = bits < 0 ? -1 : 1;
    }
    for (int s = S - 1; s >= 0; --s) {
        const int b = S - 1 - s;                                     // byte index from the bottom
        const float p2 = __int_as_float((127 + 8 * b - T) << 23);   // 2^(8b - T)
        float f[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t w = b < 4 ? lo[j] >> (8 * b) : hi[j] >> (8 * (b - 4));
            const int d = s > 0 ? (int)(w & 0xFFu) - 128 : (int)w;   // the top digit: all of W above
            f[j] = bad[j] ? __int_as_float(0x7FC00000) : (float)(sgn[j] * d) * p2;   // exact: |q| <= 2^7
        }
        uint4 w;   // every value is exact in bf16
        w.x = pack(__float2bfloat16_rn(f[0]), __float2bfloat16_rn(f[1]));
        w.y = pack(__float2bfloat16_rn(f[2]), __float2bfloat16_rn(f[3]));
        w.z = pack(__float2bfloat16_rn(f[4]), __float2bfloat16_rn(f[5]));
        w.w = pack(__float2bfloat16_rn(f[6]), __float2bfloat16_rn(f[7]));
        dst[s * pstep] = w;
    }
}

// The slicing of both operands of a product in one launch: blocks
// [0, a.gx a.gy) serve a, the rest b; blockIdx.y is the instance.
__global__ void __launch_bounds__(256) slice_pair_kernel(SliceOp a, SliceOp b) {
    __shared__ double t[64][33];   // transposed staging: t[k_local][i_local]
    const int na = a.gx * a.gy;
    const int id = (int)blockIdx.x;
    if (id < na) slice_tile(a, id % a.gx, id / a.gx, blockIdx.y, t);
    else slice_tile(b, (id - na) % b.gx, (id - na) / b.gx, blockIdx.y, t);
}

// ------------------------------------------------------------------ host side
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encode() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

bool make_map(CUtensorMap* map, const __nv_bfloat16* base, int S, int rows, int Kp, int box_rows) {
    EncodeTiled enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t elem[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, elem,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Per-device state of the engine: SM count and whether the kernel attributes
// (dynamic shared memory) have been set in that device's context.
constexpr int kMaxDevices = 64;
struct DeviceState {
    int sms = 0;
    bool attr = false;
};
std::mutex g_dev_mu;
DeviceState g_dev[kMaxDevices];

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    return dev;
}

int num_sms() {
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_dev[dev].sms) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_dev[dev].sms = sms > 0 ? sms : 1;
    }
    return g_dev[dev].sms;
}

// Dynamic shared memory of a kernel: the stages and the barriers (the final
// pass keeps its column exponents in static shared memory); the rest is L1.
size_t smem_bytes(bool lean) {
    return (lean ? LEAN_STAGES : STAGES) * STAGE_BYTES + 1024 + 256;
}

// Set the kernels' shared-memory attribute once per device; false if the
// kernel cannot launch with its block size there.
bool prepare_kernels() {
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_dev[dev].attr) return true;
    const void* kernels[3] = {(const void*)tc_gemm_kernel<false, true>, (const void*)tc_gemm_kernel<true, true>,
                              (const void*)tc_gemm_kernel<true, false>};
    for (int i = 0; i < 3; ++i) {
        const void* k = kernels[i];
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(i >= 1));
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && fa.maxThreadsPerBlock < THREADS) {
            std::fprintf(stderr, "tc_gemm: kernel uses %d registers; at most %d threads per block fit\n",
                         fa.numRegs, fa.maxThreadsPerBlock);
            return false;
        }
    }
    g_dev[dev].attr = true;
    return true;
}

}  // namespace

TcMode tc_mode(int prec) {
    TcMode m;
    if (prec == TC_BF16) { m.S = 1; m.L = 0; m.exact = 0; }
    else if (prec == TC_FP32) { m.S = 4; m.L = 3; m.exact = 1; }   // 31 bits: FP32-class or better
    else { m.S = 7; m.L = 6; m.exact = 1; }                        // 55 bits: FP64-class
    return m;
}

int tc_pairs(const TcMode& m) {
    int n = 0;
    for (int s = 0; s < m.S; ++s)
        for (int t = 0; t < m.S; ++t)
            if (s + t <= m.L) ++n;
    return n;
}

size_t tc_workspace_bytes(int M, int N, int K, const TcMode& m, int batch) {
    const size_t Kp = (size_t)((K + 7) / 8) * 8;
    auto al = [](size_t x) { return (x + 1023) & ~size_t(1023); };
    return al((size_t)batch * m.S * M * Kp * 2) + al((size_t)batch * m.S * N * Kp * 2) +
           al(8 * (size_t)batch * (M + N)) + 1024;
}

size_t tc_smem_bytes() { return smem_bytes(false); }

int tc_gemm(int M, int N, int K, const double* A, int lda, bool transA, const double* B, int ldb, bool transB,
            const Epilogue& epi, const TcMode& mode, void* ws, size_t ws_bytes, int* err, cudaStream_t st,
            int* kernels, cudaEvent_t ev_begin, cudaEvent_t ev_end, int batch, long long stride,
            bool one_tile_per_cta, bool sym_out, unsigned wait_limit) {
    if (sym_out && (M != N || epi.partials)) return -1;
    const int Kp = ((K + 7) / 8) * 8;
    if (batch < 1 || tc_workspace_bytes(M, N, K, mode, batch) > ws_bytes) return -1;
    auto al = [](size_t x) { return (x + 1023) & ~size_t(1023); };
    char* p = static_cast<char*>(ws);
    __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(p);
    p += al((size_t)batch * mode.S * M * Kp * 2);
    __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(p);
    p += al((size_t)batch * mode.S * N * Kp * 2);
    unsigned long long* ea = reinterpret_cast<unsigned long long*>(p);
    unsigned long long* eb = ea + (size_t)batch * M;

    // slices of op(A) (rows i, length K) and of op(B)^T (rows j, length K)
    if (mode.exact) {
        // per-row maxima of op(A) and of op(B)^T (= columns of op(B))
        if (cudaMemsetAsync(ea, 0, 8 * (size_t)batch * (M + N), st) != cudaSuccess) return -1;
        // both operands in one launch (the rows of op(A) and of op(B)^T)
        auto maxop = [&](int rows, const double* X, int ld, int colkind, unsigned long long* mx) {
            MaxOp o{rows, K, X, ld, colkind, mx, stride, 0, 0};
            o.gx = colkind ? (rows + 31) / 32 : (rows + 7) / 8;
            o.gy = colkind ? (K + 255) / 256 : 1;
            return o;
        };
        const MaxOp oa = maxop(M, A, lda, transA ? 1 : 0, ea), ob = maxop(N, B, ldb, transB ? 0 : 1, eb);
        absmax_pair_kernel<<<dim3(oa.gx * oa.gy + ob.gx * ob.gy, batch), 256, 0, st>>>(oa, ob);
        *kernels += 1;
    }
    {
        auto sliceop = [&](int rows, const double* X, int ld, int trans, const unsigned long long* mx,
                           __nv_bfloat16* out) {
            return SliceOp{rows, K, Kp, X, ld, trans, mode.exact ? mx : nullptr, mode.S, mode.exact, out, stride,
                           (Kp + 63) / 64, (rows + 31) / 32};
        };
        const SliceOp sa_op = sliceop(M, A, lda, transA ? 1 : 0, ea, sa);
        const SliceOp sb_op = sliceop(N, B, ldb, transB ? 0 : 1, eb, sb);
        slice_pair_kernel<<<dim3(sa_op.gx * sa_op.gy + sb_op.gx * sb_op.gy, batch), 256, 0, st>>>(sa_op, sb_op);
        *kernels += 1;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, sa, batch * mode.S, M, Kp, BM) || !make_map(&mb, sb, batch * mode.S, N, Kp, BN))
        return -1;

    TcParams P;
    P.M = M; P.N = N; P.K = K;
    P.npairs = 0;   // ordered by diagonal s + t (the epilogue sums a diagonal in int32)
    for (int d = 0; d <= mode.L; ++d)
        for (int s = 0; s < mode.S; ++s) {
            const int t = d - s;
            if (t >= 0 && t < mode.S) { P.pair_s[P.npairs] = s; P.pair_t[P.npairs] = t; ++P.npairs; }
        }
    P.exact = mode.exact;
    P.sym = sym_out ? 1 : 0;
    P.S = mode.S;
    P.batch = batch;
    P.stride = stride;
    P.chunk = mode.exact ? 1024 : ((K + BK - 1) / BK) * BK;   // 1024 * 2^14 = 2^24
    // Pairs of one diagonal share an accumulator in groups of g when the whole
    // (padded) K is one chunk: g * K_padded <= 1024 keeps every partial sum of
    // the group's products within 2^24 units.  Short products then drain once
    // per group instead of once per pair (for K = 64 once per diagonal).
    {
        const int kchunks = (K + P.chunk - 1) / P.chunk;
        const int klen = kchunks == 1 ? ((K + BK - 1) / BK) * BK : P.chunk;
        const int g = mode.exact ? std::max(1, 1024 / klen) : 1;
        P.ngroups = 0;
        for (int p0 = 0; p0 < P.npairs;) {
            const int d = P.pair_s[p0] + P.pair_t[p0];
            int p1 = p0;
            while (p1 < P.npairs && P.pair_s[p1] + P.pair_t[p1] == d) ++p1;
            for (int p = p0; p < p1; p += g) {
                P.grp_pair0[P.ngroups] = p;
                P.grp_npair[P.ngroups] = std::min(g, p1 - p);
                ++P.ngroups;
            }
            p0 = p1;
        }
    }
    // Horner in int64 up to the last diagonal d with |C| <= 1.05 K 2^(14+8d) < 2^62
    // (the sum over the diagonals is below 1.01 K 2^(14+8d); the margin also
    // covers the FP32 sums of the later diagonals, < 0.03 K 2^(14+8 dint));
    // then the largest shift h that keeps V = C 2^h + F 2^h below 2^62
    P.dint = -1;
    if (mode.exact)
        for (int d = 0; d <= mode.L; ++d)
            if (1.05 * (double)K * std::ldexp(1.0, 14 + 8 * d) < std::ldexp(1.0, 62)) P.dint = d;
    P.ubase = mode.exact ? 14 + 8 * std::max(P.dint, 0) : 0;
    P.hshift = 0;
    if (mode.exact)
        while (P.hshift < 40 && 1.05 * (double)K * std::ldexp(1.0, P.ubase + P.hshift + 1) < std::ldexp(1.0, 62))
            ++P.hshift;
    P.tiles_m = (M + BM - 1) / BM;
    P.tiles_n = (N + BN - 1) / BN;
    P.epi = epi;
    for (int o = 0; o < 3; ++o) P.okind[o] = out_kind(epi, o);
    P.err = err;
    P.wait_limit = wait_limit ? wait_limit : WAIT_LIMIT;
    P.rmax = mode.exact ? ea : nullptr;
    P.cmax = mode.exact ? eb : nullptr;
    const int tiles = sym_out ? P.tiles_m * (P.tiles_m + 1) / 2 : P.tiles_m * P.tiles_n;   // per instance
    // one K-chunk per pair (short products, or BF16 with its single pair): few
    // units per tile, so the final pass is most of a tile's latency -- the lean one
    const bool lean = (K + P.chunk - 1) / P.chunk == 1;
    if (!prepare_kernels()) return -1;
    if (ev_begin) cudaEventRecord(ev_begin, st);
    {
        const int all_tiles = tiles * batch;
        // persistent (one CTA per SM walking the tiles) unless the caller wants
        // the SMs released after every tile (so higher-priority streams get in)
        const int grid = (one_tile_per_cta || all_tiles < num_sms()) ? all_tiles : num_sms();
        if (!mode.exact) tc_gemm_kernel<true, false><<<grid, THREADS, smem_bytes(true), st>>>(ma, mb, P);
        else if (lean) tc_gemm_kernel<true, true><<<grid, THREADS, smem_bytes(true), st>>>(ma, mb, P);
        else tc_gemm_kernel<false, true><<<grid, THREADS, smem_bytes(false), st>>>(ma, mb, P);
    }
    if (ev_end) cudaEventRecord(ev_end, st);
    *kernels += 1;
    if (cudaError_t e = cudaPeekAtLastError(); e != cudaSuccess) {
        std::fprintf(stderr, "tc_gemm: launch failed: %s\n", cudaGetErrorString(e));
        return -1;
    }
    return EPI_WARPS * tiles;   // pair partials per instance: one per (tile, epilogue warp)
}

}  // namespace pinv
