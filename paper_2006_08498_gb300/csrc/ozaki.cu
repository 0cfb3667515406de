// FP64-accurate complex products H * Y on the BF16 tensor cores (tcgen05),
// by the Ozaki scheme (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 2012):
// each operand is split into S = 6 slices of BETA = 8 bits with a shared
// power-of-two scale per row of H and per column of Y, slice products are
// formed on the tensor cores, and the products are summed back in
// exact integer arithmetic where it matters.  This is the Chebyshev
// filter's product (Sec. 3 and the Supplement's "Filter" item: a repeated
// HEMM), the Rayleigh-Ritz product H Q and the Lanczos products.
//
// Representation.  With E_i = the exponent of max_k |H_ik| (|H_ik| <
// 2^E_i), X_ik = rint(H_ik 2^(48 - E_i)) is an integer with |X| <= 2^48,
// written in balanced base-256 digits t_1 .. t_6 (|t_1| <= 256, |t_p| <=
// 128 for p >= 2) so that H_ik ~ 2^E_i sum_p t_p 2^(-8p).  Slice p is stored
// as the BF16 value t_p 2^(-8p) (exact: at most 9 significant bits).  Y is
// split the same way per column j (exponent F_j), re and im sharing it.
//
// Products.  Slice pair (p, q) contributes integers times 2^(-8(p+q)).
// Every slice diagonal g = p + q is accumulated in FP32 over K chunks of 64
// only, then drained: over one chunk the partial sums of diagonal g are
// integer multiples of 2^(-8g) whose magnitude stays below 2^24 of those
// units (at most 6 products of at most 2^15 per k and per real MMA), so the
// diagonals 2..5 are exact; they are converted to integers and added into
// one 64-bit integer per output element, S = sum_g d_g 2^(8(5-g)) (|S| <
// 2^57 for K = 50000).  Diagonals 6 and 7 (weight <= 2^-32 of the leading
// one) share one FP32 accumulator per chunk, summed across chunks in an FP32
// register with round-to-nearest.  Diagonals > 7 are dropped.  Keeping
// every tensor-core accumulation to 64 terms matters: the accumulator
// truncates toward zero, so an FP32 sum over the whole K would carry a bias
// growing linearly with K.  The result is recombined in FP64:
// C_ij = 2^(E_i + F_j) (S_ij 2^-40 + T_ij).
//
// Complex arithmetic as two real MMAs per slice pair into one accumulator
// of 2w columns [re | im]:  Hr x [Yr | Yi]  +  Hi x [-Yi | Yr].
//
// Tiling: CTA = 128 rows x 24 complex columns (MMA M = 128, N = 48), K
// chunks of 64 (one 128-byte swizzle atom).  Warp 0 issues TMA loads, warp 1
// issues tcgen05.mma, warps 2..9 drain every chunk's accumulators (double
// buffered in TMEM: 2 x 5 x 48 = 480 columns) and run the epilogue.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace {

constexpr int kBeta = 8;
constexpr int kS = 6;              // slices per operand (stored)
constexpr int kBM = 128;           // rows per CTA
constexpr int kW = 24;             // complex columns per CTA
constexpr int kN = 2 * kW;         // MMA N
constexpr int kKC = 64;            // K chunk
constexpr int kAStages = 3;
constexpr int kBBufs = 2;
constexpr int kATile = kBM * kKC * 2;                 // 16 KB (one slice part)
constexpr int kAStageBytes = 2 * kATile;              // Hr_p and Hi_p
constexpr int kBPart = kW * kKC * 2;                  // 3 KB
constexpr int kBSlice = 3 * kBPart;                   // [-Yi | Yr | Yi]
constexpr int kDrainWarps = 8;
constexpr int kThreads = 64 + 32 * kDrainWarps;       // producer, MMA, drain warps
constexpr int kTmemCols = 512;
constexpr int kHalf = kN / 2;                         // columns per drain thread (re or im)

// Variants: slices 1..NSL of each operand, pairs with p + q <= NSL + 1;
// diagonals 2..EXT exact, diagonals EXT+1..NSL+1 (if any) in the FP32 tail.
// FP64 accuracy: (6, 5).  Mixed precision: (4, 5): 32 bits per operand
// relative to its row/column maximum, every diagonal exact.
template <int NSL, int EXT>
struct OzCfg {
    static constexpr int kSl = NSL;
    static constexpr int kMaxD = NSL + 1;
    static constexpr int kNEx = EXT - 1;                        // exact accumulators
    static constexpr bool kTail = EXT < NSL + 1;
    static constexpr int kSlots = kNEx + (kTail ? 1 : 0);       // accumulators per buffer
    static constexpr int kBBufBytes = kSl * kBSlice;
    static constexpr int kSmem = kAStages * kAStageBytes + kBBufs * kBBufBytes + 1024;
    static constexpr int kEx = EXT;
};
using CfgFP64 = OzCfg<6, 5>;
using CfgMixed = OzCfg<4, 5>;
static_assert(CfgFP64::kSmem <= 232448 && 2 * CfgFP64::kSlots * kN <= kTmemCols, "resources");
static_assert(CfgMixed::kSmem <= 232448 && 2 * CfgMixed::kSlots * kN <= kTmemCols, "resources");
static_assert(kN % 16 == 0 && kW % 8 == 0 && kHalf % 8 == 0, "MMA N, TMA box rows, TMEM loads");

__device__ __forceinline__ void split_digits(double x, int E, int *t) {
    // X = rint(x 2^(48 - E)), |X| <= 2^48; balanced base-256 digits
    long long X = __double2ll_rn(ldexp(x, kBeta * kS - E));
#pragma unroll
    for (int p = kS - 1; p >= 1; p--) {
        int d = (int)(X & 0xFF);
        if (d >= 128) d -= 256;
        X = (X - d) >> 8;
        t[p] = d;
    }
    t[0] = (int)X;
}

// BF16 bit pattern of v; v has at most 9 significant bits, so dropping the
// low 16 bits of its FP32 pattern is exact.
__device__ __forceinline__ uint16_t bf16_exact(float v) {
    return (uint16_t)(__float_as_uint(v) >> 16);
}

__device__ __forceinline__ float slice_value(int t, int p) {
    return (float)t * __int_as_float((127 - kBeta * (p + 1)) << 23);   // t 2^(-8(p+1))
}

// ----------------------------------------------------------- exponents
// E[i] = max over the row (rows_are_cols = 0) or column (1) of the frexp
// exponent of |re| and |im|; INT_MIN for an all-zero line.
// Non-finite entries cannot be sliced; they are reported through the
// error word (fmax alone would skip NaN).
__global__ void k_row_exponent(int64_t N, const z_t *__restrict__ H, int64_t ldh, int *E,
                               int cols_per_block, ChaseScalars *sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t k0 = (int64_t)blockIdx.y * cols_per_block;
    const int64_t k1 = (k0 + cols_per_block < N) ? k0 + cols_per_block : N;
    double mx = 0.0;
    bool finite = true;
    for (int64_t k = k0; k < k1; k++) {
        const z_t h = H[i + k * ldh];
        finite = finite && isfinite(h.x) && isfinite(h.y);
        mx = fmax(mx, fmax(fabs(h.x), fabs(h.y)));
    }
    if (!finite) set_error(sc, DEV_NONFINITE, (int)i);
    if (mx > 0.0) {
        int e;
        frexp(mx, &e);
        atomicMax(&E[i], e);
    }
}

__global__ void k_col_exponent(int64_t N, int n, const z_t *__restrict__ Y, int64_t ldy, int *F,
                               ChaseScalars *sc) {
    const int j = blockIdx.y;
    if (j >= n) return;
    double mx = 0.0;
    bool finite = true;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const z_t y = Y[k + j * ldy];
        finite = finite && isfinite(y.x) && isfinite(y.y);
        mx = fmax(mx, fmax(fabs(y.x), fabs(y.y)));
    }
    if (!finite) set_error(sc, DEV_NONFINITE, j);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) {
        int e;
        frexp(mx, &e);
        atomicMax(&F[j], e);
    }
}

__global__ void k_fill_int(int *p, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// ------------------------------------------------------------ slicing
// Slices are stored K-chunk-tiled: for matrix `part` (slice and re/im), K
// chunk kc = k / 64 holds all rows x 64 K-elements contiguously, so the
// tile a CTA loads (rows x 64) is one contiguous block of memory:
// index = ((part * nch + kc) * rows + row) * 64 + k % 64.
__host__ __device__ __forceinline__ int64_t tiled_index(int part, int64_t k, int64_t row,
                                                       int64_t Kp, int64_t rows) {
    const int64_t nch = Kp / 64;
    return (((int64_t)part * nch + k / 64) * rows + row) * 64 + (k % 64);
}

// A slices of H: slice p of re/im H_ik at tiled_index(p*2 + ri, k, i).  32 x 32 tiles through shared memory; padded rows and columns
// (>= N) are written as zeros.
__global__ void k_slice_h(int64_t N, int64_t Np, const z_t *__restrict__ H, int64_t ldh,
                          const int *__restrict__ E, uint16_t *A) {
    __shared__ z_t tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + tx, k = k0 + r;       // column k, rows i: coalesced
        tile[r][tx] = (i < N && k < N) ? H[i + k * ldh] : zmk(0.0, 0.0);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, k = k0 + tx;       // row i, consecutive k
        const z_t h = tile[tx][r];
        int e = (i < N) ? E[i] : INT_MIN;
        if (e == INT_MIN) e = 0;
        int tr[kS], ti[kS];
        split_digits(h.x, e, tr);
        split_digits(h.y, e, ti);
#pragma unroll
        for (int p = 0; p < kS; p++) {
            A[tiled_index(p * 2 + 0, k, i, Np, Np)] = bf16_exact(slice_value(tr[p], p));
            A[tiled_index(p * 2 + 1, k, i, Np, Np)] = bf16_exact(slice_value(ti[p], p));
        }
    }
}

// B slices of Y: slice q of Yr, Yi and -Yi (part 0, 1, 2) of column j at
// tiled_index(q*3 + part, k, j) with mp rows.
__global__ void k_slice_y(int64_t N, int64_t Np, int n, int mp, const z_t *__restrict__ Y,
                          int64_t ldy, const int *__restrict__ F, uint16_t *B) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (k >= Np) return;
    z_t y = zmk(0.0, 0.0);
    int e = 0;
    if (j < n && k < N) {
        y = Y[k + j * ldy];
        e = F[j] == INT_MIN ? 0 : F[j];
    }
    int tr[kS], ti[kS];
    split_digits(y.x, e, tr);
    split_digits(y.y, e, ti);
#pragma unroll
    for (int q = 0; q < kS; q++) {
        B[tiled_index(q * 3 + 0, k, j, Np, mp)] = bf16_exact(slice_value(tr[q], q));
        B[tiled_index(q * 3 + 1, k, j, Np, mp)] = bf16_exact(slice_value(ti[q], q));
        B[tiled_index(q * 3 + 2, k, j, Np, mp)] = bf16_exact(slice_value(-ti[q], q));
    }
}

// ---------------------------------------------------------- the GEMM
struct OzArgs {
    int64_t M;        // rows of the output (N)
    int n;            // complex columns of the output
    int mp;           // padded columns (multiple of kW)
    int nchunks;      // Np / kKC
    const int *E;     // row exponents of H (padded to Np)
    const int *F;     // column exponents of Y
    GemmEpi ep;
    const z_t *Y;     // FP64 operand (for the CHEB epilogue)
    int64_t ldy;
    z_t *C;
    int64_t ldc;
    ChaseScalars *sc;
    int csplit;       // K chunks per split (gridDim.z splits)
    z_t *P;           // split > 1: FP64 partial products [z][j][i], ld M
};

template <class Cfg>
__global__ void __launch_bounds__(kThreads, 1)
k_ozaki_zgemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              OzArgs args) {
    constexpr int kSl = Cfg::kSl;
    constexpr int kSlots = Cfg::kSlots;
    constexpr int kBBufBytes = Cfg::kBBufBytes;
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;                                        // kAStages x 32 KB
    uint8_t *sB = sm + kAStages * kAStageBytes;              // kBBufs x slices x 9 KB
    __shared__ uint64_t fullA[kAStages], emptyA[kAStages], fullB[kBBufs], emptyB[kBBufs];
    __shared__ uint64_t accFull[2], accEmpty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int j0 = blockIdx.x * kW;
    const int64_t i0 = (int64_t)blockIdx.y * kBM;
    const int nch = args.nchunks;
    const int c0 = blockIdx.z * args.csplit;
    const int c1 = min(nch, c0 + args.csplit);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAStages; s++) { tc::mbar_init(&fullA[s], 1); tc::mbar_init(&emptyA[s], 1); }
        for (int s = 0; s < kBBufs; s++) { tc::mbar_init(&fullB[s], 1); tc::mbar_init(&emptyB[s], 1); }
        for (int s = 0; s < 2; s++) { tc::mbar_init(&accFull[s], 1); tc::mbar_init(&accEmpty[s], kDrainWarps); }
        abort_flag = 0;
        tc::mbar_fence_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_base, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            tc::prefetch_tmap(&tmA);
            tc::prefetch_tmap(&tmB);
            int use = 0;
            for (int c = c0; c < c1 && !abort_flag; c++) {
                const int lc = c - c0, bb = lc & 1;
                if (lc >= 2 && !tc::mbar_wait(&emptyB[bb], ((lc >> 1) - 1) & 1, &abort_flag)) break;
                tc::mbar_expect_tx(&fullB[bb], kBBufBytes);
                uint8_t *bdst = sB + bb * kBBufBytes;
                for (int q = 0; q < kSl; q++) {
                    // smem [-Yi | Yr | Yi] from parts 2, 0, 1
                    tc::tma_load_3d(bdst + q * kBSlice + 0 * kBPart, &tmB, 0, j0, (q * 3 + 2) * nch + c, &fullB[bb]);
                    tc::tma_load_3d(bdst + q * kBSlice + 1 * kBPart, &tmB, 0, j0, (q * 3 + 0) * nch + c, &fullB[bb]);
                    tc::tma_load_3d(bdst + q * kBSlice + 2 * kBPart, &tmB, 0, j0, (q * 3 + 1) * nch + c, &fullB[bb]);
                }
                bool ok = true;
                for (int p = 0; p < kSl; p++, use++) {
                    const int st = use % kAStages, n = use / kAStages;
                    if (n >= 1 && !tc::mbar_wait(&emptyA[st], (n - 1) & 1, &abort_flag)) { ok = false; break; }
                    tc::mbar_expect_tx(&fullA[st], kAStageBytes);
                    uint8_t *adst = sA + st * kAStageBytes;
                    tc::tma_load_3d(adst, &tmA, 0, (int)i0, (p * 2 + 0) * nch + c, &fullA[st]);
                    tc::tma_load_3d(adst + kATile, &tmA, 0, (int)i0, (p * 2 + 1) * nch + c, &fullA[st]);
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(kBM, kN);
            int use = 0;
            for (int c = c0; c < c1 && !abort_flag; c++) {
                const int lc = c - c0, bb = lc & 1;
                if (!tc::mbar_wait(&fullB[bb], (lc >> 1) & 1, &abort_flag)) break;
                if (lc >= 2 && !tc::mbar_wait(&accEmpty[bb], ((lc >> 1) - 1) & 1, &abort_flag)) break;
                tc::fence_after();
                bool started[kSlots];
#pragma unroll
                for (int s = 0; s < kSlots; s++) started[s] = false;
                const uint8_t *bsrc = sB + bb * kBBufBytes;
                bool ok = true;
                for (int p = 1; p <= kSl; p++, use++) {
                    const int st = use % kAStages, n = use / kAStages;
                    if (!tc::mbar_wait(&fullA[st], n & 1, &abort_flag)) { ok = false; break; }
                    tc::fence_after();
                    const uint8_t *aR = sA + st * kAStageBytes, *aI = aR + kATile;
                    const uint64_t a_r = tc::sdesc_sw128(aR), a_i = tc::sdesc_sw128(aI);
                    for (int q = 1; p + q <= Cfg::kMaxD; q++) {
                        const int g = p + q;
                        const int slot = (g <= Cfg::kEx) ? g - 2 : kSlots - 1;
                        const uint32_t d = tmem + (uint32_t)((bb * kSlots + slot) * kN);
                        const bool acc0 = started[slot];
                        started[slot] = true;
                        const uint8_t *bq = bsrc + (q - 1) * kBSlice;
                        const uint64_t b_pos = tc::sdesc_sw128(bq + kBPart);   // [Yr | Yi]
                        const uint64_t b_neg = tc::sdesc_sw128(bq);            // [-Yi | Yr]
#pragma unroll
                        for (int kk = 0; kk < kKC / 16; kk++) {
                            tc::mma_bf16(d, a_r + 2 * kk, b_pos + 2 * kk, idesc, (acc0 || kk > 0) ? 1u : 0u);
                            tc::mma_bf16(d, a_i + 2 * kk, b_neg + 2 * kk, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&emptyA[st]);
                }
                if (!ok) break;
                tc::mma_commit(&emptyB[bb]);
                tc::mma_commit(&accFull[bb]);
            }
        }
    } else {
        // ------------------------------------------------ drain + epilogue
        // warp w: TMEM lanes of quadrant (w & 3); columns [half*24, half*24+24)
        // of every accumulator (half 0: re, half 1: im).
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        long long S[kHalf];
        float T[kHalf];
#pragma unroll
        for (int j = 0; j < kHalf; j++) { S[j] = 0; T[j] = 0.f; }
        bool ok = true;
        for (int c = c0; c < c1; c++) {
            const int lc = c - c0, bb = lc & 1;
            if (!tc::mbar_wait(&accFull[bb], (lc >> 1) & 1, &abort_flag)) { ok = false; break; }
            tc::fence_after();
#pragma unroll
            for (int g = 2; g <= Cfg::kEx; g++) {
                const float scale = __int_as_float((127 + kBeta * g) << 23);   // 2^(8g)
                const int shift = kBeta * (5 - g);                             // S in units of 2^-40
                const uint32_t col = (uint32_t)((bb * kSlots + (g - 2)) * kN + half * kHalf);
                uint32_t r[kHalf];
#pragma unroll
                for (int h = 0; h < kHalf; h += 8) tc::tmem_ld8(tmem + lane_addr + col + h, r + h);
                tc::tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < kHalf; u++) {
                    const int d = __float2int_rn(__uint_as_float(r[u]) * scale);
                    S[u] += (long long)d << shift;
                }
            }
            if (Cfg::kTail) {
                const uint32_t col = (uint32_t)((bb * kSlots + kSlots - 1) * kN + half * kHalf);
                uint32_t r[kHalf];
#pragma unroll
                for (int h = 0; h < kHalf; h += 8) tc::tmem_ld8(tmem + lane_addr + col + h, r + h);
                tc::tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < kHalf; u++) T[u] += __uint_as_float(r[u]);
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&accEmpty[bb]);
        }
        if (ok) {
            const int64_t i = i0 + row;
            if (i < args.M) {
                int e = args.E[i];
                if (e == INT_MIN) e = 0;
#pragma unroll
                for (int u = 0; u < kHalf; u++) {
                    const int j = j0 + u;
                    if (j >= args.n) continue;
                    int f = args.F[j];
                    if (f == INT_MIN) f = 0;
                    const double v = ldexp((double)S[u] * 0x1.0p-40 + (double)T[u], e + f);
                    double out = v;
                    if (args.P) {        // split-K partial; summed and finished by k_split_reduce
                        double *pp = (double *)(args.P + ((int64_t)blockIdx.z * args.n + j) * args.M + i);
                        pp[half] = out;
                        continue;
                    }
                    if (args.ep.mode == GEMM_CHEB) {
                        const double y = half ? args.Y[i + j * args.ldy].y : args.Y[i + j * args.ldy].x;
                        out = args.ep.s1 * (v - args.ep.c * y);
                        if (args.ep.Yp) {
                            const z_t yp = args.ep.Yp[i + j * args.ep.ldyp];
                            out -= args.ep.s2 * (half ? yp.y : yp.x);
                        }
                    }
                    double *cp = (double *)(args.C + i + j * args.ldc);
                    cp[half] = out;
                }
            }
        }
    }

    tc::fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) set_error(args.sc, DEV_TIMEOUT, blockIdx.y * gridDim.x + blockIdx.x);
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// C = epi(sum over splits z of P[z]) in increasing z (deterministic).
__global__ void k_split_reduce(int64_t M, int n, int nsplit, const z_t *__restrict__ P,
                               GemmEpi ep, const z_t *__restrict__ Y, int64_t ldy, z_t *C,
                               int64_t ldc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= M) return;
    z_t v = zmk(0.0, 0.0);
    for (int z = 0; z < nsplit; z++) v = zadd(v, P[((int64_t)z * n + j) * M + i]);
    if (ep.mode == GEMM_CHEB) {
        v = zscale(zsub(v, zscale(Y[i + j * ldy], ep.c)), ep.s1);
        if (ep.Yp) v = zsub(v, zscale(ep.Yp[i + j * ep.ldyp], ep.s2));
    }
    C[i + j * ldc] = v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3-D BF16 tensor of K-chunk tiles [tiles][rows][64], box 64 x box_rows x 1,
// 128-byte swizzle (the shared-memory image of one K-major rows x 64 tile).
bool make_map(CUtensorMap *m, void *base, uint64_t rows, uint64_t tiles, uint32_t box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {64, rows, tiles};
    cuuint64_t strides[2] = {64 * 2, rows * 64 * 2};
    cuuint32_t box[3] = {64, box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int64_t ozaki_padded(int64_t N) { return (N + 127) / 128 * 128; }

size_t ozaki_a_bytes(int64_t N) {
    const int64_t Np = ozaki_padded(N);
    return (size_t)kS * 2 * Np * Np * 2;
}

size_t ozaki_b_bytes(int64_t N, int m) {
    const int64_t Np = ozaki_padded(N);
    const int mp = (m + kW - 1) / kW * kW;
    return (size_t)kS * 3 * mp * Np * 2;
}

cudaError_t ozaki_prepare_h(int64_t N, const z_t *H, int64_t ldh, OzakiH *oh, ChaseScalars *sc,
                            cudaStream_t st) {
    const int64_t Np = ozaki_padded(N);
    oh->N = N;
    oh->Np = Np;
    k_fill_int<<<(unsigned)((Np + 255) / 256), 256, 0, st>>>(oh->E, (int)Np, INT_MIN);
    bse_count_launches(1);
    const int cpb = 256;
    dim3 g1((unsigned)((N + 255) / 256), (unsigned)((N + cpb - 1) / cpb));
    k_row_exponent<<<g1, 256, 0, st>>>(N, H, ldh, oh->E, cpb, sc);
    bse_count_launches(1);
    dim3 g2((unsigned)(Np / 32), (unsigned)(Np / 32));
    k_slice_h<<<g2, dim3(32, 8), 0, st>>>(N, Np, H, ldh, oh->E, (uint16_t *)oh->A);
    bse_count_launches(1);
    if (!make_map((CUtensorMap *)oh->tmap, oh->A, (uint64_t)Np, (uint64_t)(kS * 2 * (Np / kKC)),
                  kBM))
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_variant(const CUtensorMap &tmA, const CUtensorMap &tmB, const OzArgs &a,
                           dim3 grid, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_ozaki_zgemm<Cfg>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_ozaki_zgemm<Cfg><<<grid, kThreads, Cfg::kSmem, st>>>(tmA, tmB, a);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t ozaki_zgemm(const OzakiH &oh, int n, const z_t *Y, int64_t ldy, z_t *C, int64_t ldc,
                        const GemmEpi &ep, void *bslices, int *F, ChaseScalars *sc, int low,
                        z_t *partials, size_t partial_bytes, int sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t N = oh.N, Np = oh.Np;
    const int mp = (n + kW - 1) / kW * kW;
    k_fill_int<<<(mp + 255) / 256, 256, 0, st>>>(F, mp, INT_MIN);
    bse_count_launches(1);
    dim3 ge((unsigned)std::min<int64_t>((N + 255) / 256, 16), (unsigned)n);
    k_col_exponent<<<ge, 256, 0, st>>>(N, n, Y, ldy, F, sc);
    bse_count_launches(1);
    dim3 gs((unsigned)((Np + 255) / 256), (unsigned)mp);
    k_slice_y<<<gs, 256, 0, st>>>(N, Np, n, mp, Y, ldy, F, (uint16_t *)bslices);
    bse_count_launches(1);
    CUtensorMap tmB;
    if (!make_map(&tmB, bslices, (uint64_t)mp, (uint64_t)(kS * 3 * (Np / kKC)), kW))
        return cudaErrorInvalidValue;
    OzArgs a;
    a.M = N;
    a.n = n;
    a.mp = mp;
    a.nchunks = (int)(Np / kKC);
    a.E = oh.E;
    a.F = F;
    a.ep = ep;
    a.Y = Y;
    a.ldy = ldy;
    a.C = C;
    a.ldc = ldc;
    a.sc = sc;
    // split K so that the CTAs fill whole waves of the SMs: the smallest
    // ceil(tiles * s / sms) / s over s, with at least 16 K chunks per split
    // and the partials bounded by the workspace
    const int tiles = (mp / kW) * (int)(Np / kBM);
    int best = 1;
    double best_t = 1e30;
    for (int sp = 1; sp <= 16; sp++) {
        if ((int64_t)sp * 16 > a.nchunks && sp > 1) break;
        if ((int64_t)sp * n * N * (int64_t)sizeof(z_t) > partial_bytes && sp > 1) break;
        const double t = (double)((tiles * sp + sms - 1) / sms) / sp * (1.0 + 0.01 * (sp - 1));
        if (t < best_t - 1e-12) { best_t = t; best = sp; }
    }
    a.csplit = (a.nchunks + best - 1) / best;
    const int nsplit = (a.nchunks + a.csplit - 1) / a.csplit;
    a.P = (nsplit > 1) ? partials : nullptr;
    dim3 grid((unsigned)(mp / kW), (unsigned)(Np / kBM), (unsigned)nsplit);
    const CUtensorMap &tmA = *(const CUtensorMap *)oh.tmap;
    cudaError_t e = low ? launch_variant<CfgMixed>(tmA, tmB, a, grid, st)
                        : launch_variant<CfgFP64>(tmA, tmB, a, grid, st);
    if (e != cudaSuccess || nsplit == 1) return e;
    dim3 gr((unsigned)((N + 255) / 256), (unsigned)n);
    k_split_reduce<<<gr, 256, 0, st>>>(N, n, nsplit, partials, ep, Y, ldy, C, ldc);
    bse_count_launches(1);
    return cudaGetLastError();
}
