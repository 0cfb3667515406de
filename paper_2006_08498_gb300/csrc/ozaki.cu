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
// as the BF16 value t_p 2^(-8p) (exact: at most 8 significant bits).  Y is
// split the same way per column j (exponent F_j), re and im sharing it.
//
// Products.  Slice pair (p, q) contributes integers times 2^(-8(p+q)).
// The diagonals g = 2..5 are accumulated in FP32 over one or two K chunks of
// 64 only (drain_period), then drained: over that range the partial sums of
// diagonal g are integer multiples of 2^(-8g) whose magnitude stays below
// 2^24 of those units (diag_bound), so they are exact; they are converted to
// integers and added into one 64-bit integer per output element,
// S = sum_g d_g 2^(8(5-g)) (|S| < 2^57 for K = 50000).
// Keeping these accumulations to 64 terms matters: the tensor core's FP32
// accumulator truncates toward zero, so a sum over the whole K would carry a
// bias growing with K.  Diagonals 6 and 7 (weight <= 2^-32 of the leading
// one) share one FP32 accumulator over the K chunks of one work unit (at most
// kUnitChunks), whose sums over K splits are added in FP32 by the reduction:
// within a unit the truncation error is at most one FP32 ulp of the running
// tail sum per K step of 16.  Diagonals > 7 are dropped.  The result is recombined in
// FP64, C_ij = 2^(E_i + F_j) (S_ij 2^-40 + T_ij), after the K splits' S and T
// are summed (exactly, for S) by the reduction kernels.
//
// Complex arithmetic as two real MMAs per slice pair into one accumulator
// of 2w columns [re | im]:  Hr x [Yr | Yi]  +  Hi x [-Yi | Yr].
//
// Tiling: CTA = 128 rows x 48 complex columns (MMA M = 128, N = 96), K
// chunks of 64 (one 128-byte swizzle atom).  Warp 0 issues TMA loads, warp 1
// issues tcgen05.mma, warps 2..9 drain the exact accumulators and store the
// raw partials.  TMEM holds five 96-column accumulators (480 of 512
// columns): one per exact diagonal and the tail.  An MMA costs a fixed ~45
// cycles plus N/2 on this tensor core, so the widest N that leaves room for
// five accumulators is the one used; and every instruction the single MMA
// thread issues between MMAs (a barrier wait, a commit) costs issue time, so
// the pipeline is built to need few of them.
#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "gen_element.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace {

constexpr int kBeta = 8;
constexpr int kS = 6;              // slices per operand (stored)
constexpr int kBM = 128;           // rows per CTA
constexpr int kW = 48;             // complex columns per CTA
constexpr int kN = 2 * kW;         // MMA N
constexpr int kKC = 64;            // K chunk
constexpr int kAStages = 6;        // A tiles of one part (Re or Im of one slice)
constexpr int kAPairs = kAStages / 2;  // stages of one slice (Re and Im tiles, one barrier)
constexpr int kATile = kBM * kKC * 2;                 // 16 KB
constexpr int kBPart = kW * kKC * 2;                  // 6 KB
constexpr int kBSlice = 3 * kBPart;                   // [-Yi | Yr | Yi]
constexpr int kDrainWarps = 8;
constexpr int kThreads = 64 + 32 * kDrainWarps;       // producer, MMA, drain warps
constexpr int kTmemCols = 512;
constexpr int kHalf = kN / 2;                         // columns per drain thread (re or im)

// Variants: slices 1..NSL of each operand, pairs with p + q <= NSL + 1;
// diagonals 2..EXT exact, diagonals EXT+1..NSL+1 (if any) in the FP32 tail.
// FP64 accuracy: (6, 5).  The mixed precision mode's cheaper levels: (4, 5),
// 32 bits per operand relative to its row/column maximum, every diagonal
// exact; (5, 5), 40 bits, diagonal 6 in the tail.
template <int NSL, int EXT, bool TRI = false>
struct OzCfg {
    static constexpr int kSl = NSL;
    static constexpr bool kTri = TRI;        // half storage of H's slices
    static constexpr bool kTail = EXT < NSL + 1;
    static constexpr int kAcc = (EXT - 1) + (kTail ? 1 : 0);     // TMEM accumulators
    static constexpr int kSmem = kAStages * kATile + (NSL + 1) * kBSlice + 1024;
    static constexpr int kEx = EXT;
};
using CfgFP64 = OzCfg<6, 5>;
using CfgMixed = OzCfg<4, 5>;
using CfgMid = OzCfg<5, 5>;
using CfgFP64Tri = OzCfg<6, 5, true>;
using CfgMixedTri = OzCfg<4, 5, true>;
using CfgMidTri = OzCfg<5, 5, true>;
static_assert(CfgFP64::kSmem <= 232448 && CfgFP64::kAcc * kN <= kTmemCols, "resources");
static_assert(CfgMixed::kSmem <= 232448 && CfgMixed::kAcc * kN <= kTmemCols, "resources");
static_assert(CfgMid::kSmem <= 232448 && CfgMid::kAcc * kN <= kTmemCols, "resources");
static_assert(kN % 16 == 0 && kW % 8 == 0 && kHalf % 16 == 0, "MMA N, TMA box rows, TMEM loads");
static_assert(kBPart % 1024 == 0 && kATile % 1024 == 0, "128-byte swizzle atoms stay 1024-aligned");

// rint(x 2^sh), ties to even, for a finite x with |x 2^sh| < 2^62, from the
// bit pattern of x with integer operations only (FP64 issue is scarce on
// this part, the integer pipes are not).  x = mant 2^ex exactly.
__device__ __forceinline__ long long scaled_rint(double x, int sh) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    int ex = -1074;                                 // subnormal or zero
    if (ef != 0) {
        mant |= 1ull << 52;
        ex = ef - 1075;
    }
    const int s = ex + sh;
    unsigned long long q;
    if (s >= 0) {
        q = mant << s;
    } else if (-s > 54) {
        q = 0;                                      // mant < 2^53: below one half
    } else {
        const int r = -s;
        q = mant >> r;
        const unsigned long long rem = mant & ((1ull << r) - 1), half = 1ull << (r - 1);
        q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

// Largest |re| or |im| of a line as a bit pattern: for non-negative doubles
// the integer order of the patterns is the numeric order, and any Inf or NaN
// compares above kNonFinite.
constexpr unsigned long long kNonFinite = 0x7FF0000000000000ull;
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// frexp exponent of the value with pattern mb (finite, non-zero)
__device__ __forceinline__ int frexp_bits(unsigned long long mb) {
    int e;
    frexp(__longlong_as_double((long long)mb), &e);
    return e;
}

__device__ __forceinline__ void split_digits(double x, int E, int *t) {
    // X = rint(x 2^(48 - E)), |X| <= 2^48 since |x| < 2^E; balanced base-256 digits
    long long X = scaled_rint(x, kBeta * kS - E);
#pragma unroll
    for (int p = kS - 1; p >= 1; p--) {
        int d = (int)(X & 0xFF);
        if (d >= 128) d -= 256;
        X = (X - d) >> 8;
        t[p] = d;
    }
    t[0] = (int)X;
}

// BF16 bit pattern of v; v has at most 8 significant bits, so dropping the
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
__global__ void k_row_exponent(int64_t M, int64_t K, const z_t *__restrict__ H, int64_t ldh,
                               int *E, int cols_per_block, ChaseScalars *sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t k0 = (int64_t)blockIdx.y * cols_per_block;
    const int64_t k1 = (k0 + cols_per_block < K) ? k0 + cols_per_block : K;
    unsigned long long mb = 0;
    for (int64_t k = k0; k < k1; k++) {
        const z_t h = H[i + k * ldh];
        mb = max(mb, max(abs_bits(h.x), abs_bits(h.y)));
    }
    if (mb >= kNonFinite) set_error(sc, DEV_NONFINITE, (int)i);
    else if (mb > 0) atomicMax(&E[i], frexp_bits(mb));
}

// With rs, the exponents are those of rs[k] Y[k, j] (half storage: T Y).
__global__ void k_col_exponent(int64_t N, int n, const z_t *__restrict__ Y, int64_t ldy, int *F,
                               ChaseScalars *sc, const double *__restrict__ rs = nullptr) {
    const int j = blockIdx.y;
    if (j >= n) return;
    unsigned long long mb = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const z_t y = rs ? zscale(Y[k + j * ldy], rs[k]) : Y[k + j * ldy];
        mb = max(mb, max(abs_bits(y.x), abs_bits(y.y)));
    }
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if ((threadIdx.x & 31) == 0) {
        if (mb >= kNonFinite) set_error(sc, DEV_NONFINITE, j);
        else if (mb > 0) atomicMax(&F[j], frexp_bits(mb));
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

// A slices of an M x K matrix H (rows padded to Mp, K to Kp): slice p of
// re/im H_ik at tiled_index(p*2 + ri, k, i, Kp, Mp).  32 x 32 tiles through
// shared memory; padded rows and columns are written as zeros.
__global__ void k_slice_h(int64_t M, int64_t Mp, int64_t K, int64_t Kp,
                          const z_t *__restrict__ H, int64_t ldh, const int *__restrict__ E,
                          uint16_t *A) {
    __shared__ z_t tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + tx, k = k0 + r;       // column k, rows i: coalesced
        tile[r][tx] = (i < M && k < K) ? H[i + k * ldh] : zmk(0.0, 0.0);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, k = k0 + tx;       // row i, consecutive k
        const z_t h = tile[tx][r];
        int e = (i < M) ? E[i] : INT_MIN;
        if (e == INT_MIN) e = 0;
        int tr[kS], ti[kS];
        split_digits(h.x, e, tr);
        split_digits(h.y, e, ti);
#pragma unroll
        for (int p = 0; p < kS; p++) {
            A[tiled_index(p * 2 + 0, k, i, Kp, Mp)] = bf16_exact(slice_value(tr[p], p));
            A[tiled_index(p * 2 + 1, k, i, Kp, Mp)] = bf16_exact(slice_value(ti[p], p));
        }
    }
}

// A slices of op(A) = A^H for a K x M matrix A: op(A)_ik = conj(A_ki), read
// down column i of A (coalesced in k); exponents E[i] are those of column i.
__global__ void k_slice_ah(int64_t M, int64_t Mp, int64_t K, int64_t Kp,
                           const z_t *__restrict__ A, int64_t lda, const int *__restrict__ E,
                           uint16_t *S) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = blockIdx.y;
    if (k >= Kp || i >= Mp) return;
    z_t a = zmk(0.0, 0.0);
    int e = 0;
    if (i < M && k < K) {
        a = A[k + i * lda];
        e = E[i] == INT_MIN ? 0 : E[i];
    }
    int tr[kS], ti[kS];
    split_digits(a.x, e, tr);
    split_digits(-a.y, e, ti);
#pragma unroll
    for (int p = 0; p < kS; p++) {
        S[tiled_index(p * 2 + 0, k, i, Kp, Mp)] = bf16_exact(slice_value(tr[p], p));
        S[tiled_index(p * 2 + 1, k, i, Kp, Mp)] = bf16_exact(slice_value(ti[p], p));
    }
}

// B slices of Y: slice q of Yr, Yi and -Yi (part 0, 1, 2) of column j at
// tiled_index(q*3 + part, k, j) with mp rows.  With rs: the slices of
// rs[k] Y[k, j] (half storage: T Y).
__global__ void k_slice_y(int64_t N, int64_t Np, int n, int mp, const z_t *__restrict__ Y,
                          int64_t ldy, const int *__restrict__ F, uint16_t *B,
                          const double *__restrict__ rs = nullptr) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (k >= Np) return;
    z_t y = zmk(0.0, 0.0);
    int e = 0;
    if (j < n && k < N) {
        y = rs ? zscale(Y[k + j * ldy], rs[k]) : Y[k + j * ldy];
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

// ---------------------------------------------- half storage of H's slices
// H = T S T with T = diag(t_i), t_i = sqrt(M_i) (1 + 2^-20), M_i = max_k
// max(|Re H_ik|, |Im H_ik|): S is Hermitian and |S_ik| <= min(M_i, M_k) /
// (t_i t_k) < 1, so every row of S is sliced against the one exponent 0 and
// the digits of S_ki are those of S_ik conjugated.  Only the lower-triangle
// tiles of S are stored; H Y = T (S (T Y)).

// Row maxima M_i (bit patterns) from the lower triangle: element (i, k),
// k <= i, counts for row i and, as H_ki = conj(H_ik), for row k.  One
// 32 x 32 tile (ti >= tj) per CTA; Mx zeroed before.
__global__ void __launch_bounds__(256)
k_tri_rowmax(int64_t N, const z_t *__restrict__ H, int64_t ldh, unsigned long long *Mx) {
    const int ti = blockIdx.x, tj = blockIdx.y;
    if (ti < tj) return;
    __shared__ unsigned long long rmax[32], cmax[32];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    if (ty == 0) rmax[tx] = cmax[tx] = 0ull;
    __syncthreads();
    const int64_t i = (int64_t)ti * 32 + tx;
    unsigned long long mine = 0;
    for (int c = ty; c < 32; c += 8) {
        const int64_t k = (int64_t)tj * 32 + c;
        if (i >= N || k >= N || k > i) continue;
        const z_t h = H[i + k * ldh];
        const unsigned long long mb = max(abs_bits(h.x), abs_bits(h.y));
        mine = max(mine, mb);
        atomicMax(&cmax[c], mb);
    }
    atomicMax(&rmax[tx], mine);
    __syncthreads();
    if (ty == 0) {
        const int64_t r0 = (int64_t)ti * 32 + tx, r1 = (int64_t)tj * 32 + tx;
        if (r0 < N && rmax[tx]) atomicMax(&Mx[r0], rmax[tx]);
        if (r1 < N && cmax[tx]) atomicMax(&Mx[r1], cmax[tx]);
    }
}

// t_i, s_i = 1 / t_i (1 for an all-zero or padded row) and E_i = 0
// (INT_MIN for padded rows).  Mx may alias s (each thread reads its own
// entry before writing it).  Non-finite rows set DEV_NONFINITE.
__global__ void k_tri_scales(int64_t N, int64_t Np, const unsigned long long *Mx, double *t,
                             double *s, int *E, ChaseScalars *sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Np) return;
    double ti = 1.0;
    if (i < N) {
        const unsigned long long mb = Mx[i];
        if (mb >= kNonFinite) set_error(sc, DEV_NONFINITE, (int)i);
        else if (mb > 0) ti = sqrt(__longlong_as_double((long long)mb)) * (1.0 + 0x1.0p-20);
    }
    t[i] = ti;
    s[i] = 1.0 / ti;
    E[i] = i < N ? 0 : INT_MIN;
}

// Offset of element (row r, column c) of stored tile `slot` of part `part`
// (128 x 64, row-major).
__host__ __device__ __forceinline__ int64_t tri_index(int part, int64_t slot, int64_t nslots, int r, int c) {
    return ((part * nslots + slot) * kBM + r) * kKC + c;
}

// Slices of S into the stored tiles: tile (b, kc) of 128 rows x 64 columns,
// kc <= 2 b + 1, is slot b (b + 1) + kc of each part (Re and Im of slice p:
// parts 2p and 2p + 1).  The elements above the diagonal (in the tiles that
// straddle it) are the conjugates of their mirrors, so the strict upper
// triangle of H is never read; zeros outside N.  32 x 32 tiles through
// shared memory (tk: column tile, ti: row tile), coalesced both ways.
__global__ void __launch_bounds__(256)
k_slice_tri(int64_t N, const z_t *__restrict__ H, int64_t ldh, const double *__restrict__ s,
            int64_t nslots, uint16_t *A) {
    const int tk = blockIdx.x, ti = blockIdx.y;
    const int b = ti / (kBM / 32), kc = tk / (kKC / 32);
    if (kc > 2 * b + 1) return;
    __shared__ z_t tile[32][33];                   // tile[c][r] = S(i0 + r, k0 + c)
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t i0 = (int64_t)ti * 32, k0 = (int64_t)tk * 32;
    for (int c = ty; c < 32; c += 8) {
        const int64_t i = i0 + tx, k = k0 + c;
        z_t h = zmk(0.0, 0.0);
        if (i < N && k < N) {
            h = (k <= i) ? H[i + k * ldh] : zconj(H[k + i * ldh]);
            h = zscale(h, s[i] * s[k]);
        }
        tile[c][tx] = h;
    }
    __syncthreads();
    const int64_t slot = (int64_t)b * (b + 1) + kc;
    for (int r = ty; r < 32; r += 8) {
        const z_t h = tile[tx][r];                 // S(i0 + r, k0 + tx)
        const int row = (int)(i0 + r - (int64_t)b * kBM), col = (int)(k0 + tx - (int64_t)kc * kKC);
        int tr[kS], tim[kS];
        split_digits(h.x, 0, tr);
        split_digits(h.y, 0, tim);
#pragma unroll
        for (int p = 0; p < kS; p++) {
            A[tri_index(2 * p, slot, nslots, row, col)] = bf16_exact(slice_value(tr[p], p));
            A[tri_index(2 * p + 1, slot, nslots, row, col)] = bf16_exact(slice_value(tim[p], p));
        }
    }
}

// ------------------------------- slices of the synthetic H, H not stored
// The synthetic Hamiltonian's elements generated straight into the slices of
// H (bse_element, the generator's own element function, so the values are
// bit for bit those of bse_build_hamiltonian): the N x N complex128 matrix is
// never stored.  Two passes over the lower-triangle 32 x 32 tiles of the
// padded Np x Np matrix: the row exponents (each element counts for its row
// and, conjugated, for its column's row), then the slices of every tile and
// of its mirror.  The tables (dE, u = e^{i theta}, a, Kt) come from the
// generator's table pass.
constexpr int kGT = 32;

// Stage the a rows, u and dE of the tile's rows i0.. and columns j0..
__device__ __forceinline__ void stage_tile(int i0, int j0, int N, int R, const z_t *__restrict__ a,
                                           const z_t *__restrict__ u, const double *__restrict__ dE,
                                           z_t *sai, z_t *saj, z_t *ui, z_t *uj, double *dEi) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int e = ty * kGT + tx; e < kGT * R; e += kGT * 8) {
        const int t = e / R, r = e % R;
        sai[r * kGT + t] = (i0 + t < N) ? a[(int64_t)(i0 + t) * R + r] : zmk(0.0, 0.0);
        saj[r * kGT + t] = (j0 + t < N) ? a[(int64_t)(j0 + t) * R + r] : zmk(0.0, 0.0);
    }
    if (ty == 0) {
        ui[tx] = (i0 + tx < N) ? u[i0 + tx] : zmk(0.0, 0.0);
        uj[tx] = (j0 + tx < N) ? u[j0 + tx] : zmk(0.0, 0.0);
        dEi[tx] = (i0 + tx < N) ? dE[i0 + tx] : 0.0;
    }
}

// Row exponents: E[i] = frexp exponent of max_k max(|Re H_ik|, |Im H_ik|);
// with Mx (half storage) the maxima themselves, as bit patterns.
__global__ void __launch_bounds__(256)
k_gen_row_exponent(int Nk, int nb, int N, BseModel md, const double *__restrict__ dE,
                   const z_t *__restrict__ u, const z_t *__restrict__ a,
                   const double *__restrict__ Kt, int *E, ChaseScalars *sc,
                   unsigned long long *Mx) {
    const int ti = blockIdx.x, tj = blockIdx.y;
    if (ti < tj) return;
    extern __shared__ z_t gsm[];
    __shared__ z_t ui[kGT], uj[kGT];
    __shared__ double dEi[kGT];
    __shared__ unsigned long long rmax[kGT], cmax[kGT];
    const int R = md.rank_x;
    z_t *sai = gsm, *saj = gsm + kGT * R;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = ti * kGT, j0 = tj * kGT;
    if (ty == 0) rmax[tx] = cmax[tx] = 0ull;
    stage_tile(i0, j0, N, R, a, u, dE, sai, saj, ui, uj, dEi);
    __syncthreads();
    const int I = i0 + tx;
    unsigned long long mine = 0;
    for (int c = ty; c < kGT; c += 8) {
        const int J = j0 + c;
        if ((ti == tj && tx < c) || I >= N || J >= N) continue;
        const z_t h = bse_element(I, J, R, sai + tx, saj + c, kGT, ui[tx], uj[c], dEi[tx], Nk, nb,
                                  md.w0, Kt);
        const unsigned long long mb = max(abs_bits(h.x), abs_bits(h.y));
        mine = max(mine, mb);
        atomicMax(&cmax[c], mb);                   // row J of H holds conj(h)
    }
    atomicMax(&rmax[tx], mine);
    __syncthreads();
    if (ty == 0) {
        const unsigned long long m[2] = {rmax[tx], cmax[tx]};
        const int row[2] = {i0 + tx, j0 + tx};
        for (int k = 0; k < 2; k++) {
            if (row[k] >= N || m[k] == 0) continue;
            if (Mx) atomicMax(&Mx[row[k]], m[k]);      // k_tri_scales checks finiteness
            else if (m[k] >= kNonFinite) set_error(sc, DEV_NONFINITE, row[k]);
            else atomicMax(&E[row[k]], frexp_bits(m[k]));
        }
    }
}

// Slices of the tile (rows i0.., columns j0..) and of its mirror (rows j0..,
// columns i0.., conjugated), in the layout of k_slice_h; zeros outside N.
__global__ void __launch_bounds__(256)
k_gen_slice(int Nk, int nb, int N, int64_t Np, BseModel md, const double *__restrict__ dE,
            const z_t *__restrict__ u, const z_t *__restrict__ a, const double *__restrict__ Kt,
            const int *__restrict__ E, uint16_t *A) {
    const int ti = blockIdx.x, tj = blockIdx.y;
    if (ti < tj) return;
    extern __shared__ z_t gsm[];
    __shared__ z_t tile[kGT][kGT + 1];             // tile[r][c] = H(i0 + r, j0 + c)
    __shared__ z_t ui[kGT], uj[kGT];
    __shared__ double dEi[kGT];
    const int R = md.rank_x;
    z_t *sai = gsm, *saj = gsm + kGT * R;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = ti * kGT, j0 = tj * kGT;
    const bool diag = ti == tj;
    stage_tile(i0, j0, N, R, a, u, dE, sai, saj, ui, uj, dEi);
    __syncthreads();
    const int I = i0 + tx;
    for (int c = ty; c < kGT; c += 8) {
        const int J = j0 + c;
        z_t h = zmk(0.0, 0.0);
        if (!(diag && tx < c) && I < N && J < N)
            h = bse_element(I, J, R, sai + tx, saj + c, kGT, ui[tx], uj[c], dEi[tx], Nk, nb, md.w0,
                            Kt);
        tile[tx][c] = h;
    }
    __syncthreads();
    if (diag)                                      // the upper half of a diagonal tile
        for (int c = ty; c < kGT; c += 8)
            if (tx < c) tile[tx][c] = zconj(tile[c][tx]);
    __syncthreads();
    // direct part: row i0 + r, columns j0 + tx (consecutive K: coalesced);
    // mirror part (off-diagonal tiles): row j0 + r, columns i0 + tx
    for (int pass = 0; pass < (diag ? 1 : 2); pass++) {
        const int r0 = pass == 0 ? i0 : j0, k0 = pass == 0 ? j0 : i0;
        for (int r = ty; r < kGT; r += 8) {
            const int64_t i = r0 + r, k = k0 + tx;
            const z_t h = pass == 0 ? tile[r][tx] : zconj(tile[tx][r]);
            int e = (i < N) ? E[i] : INT_MIN;
            if (e == INT_MIN) e = 0;
            int tr[kS], tim[kS];
            split_digits(h.x, e, tr);
            split_digits(h.y, e, tim);
#pragma unroll
            for (int p = 0; p < kS; p++) {
                A[tiled_index(p * 2 + 0, k, i, Np, Np)] = bf16_exact(slice_value(tr[p], p));
                A[tiled_index(p * 2 + 1, k, i, Np, Np)] = bf16_exact(slice_value(tim[p], p));
            }
        }
    }
}

// Half storage of the synthetic H, H not stored: the slices of S = D H D
// (k_slice_tri's layout) with the elements generated.  Sub-tile (ti, tk) of
// 32 x 32 is computed from the lower tile of its pair, L = H(hi.., lo..), hi
// = max(ti, tk), lo = min(ti, tk): directly below the diagonal, conjugated
// and transposed above it.
__global__ void __launch_bounds__(256)
k_gen_slice_tri(int Nk, int nb, int N, BseModel md, const double *__restrict__ dE,
                const z_t *__restrict__ u, const z_t *__restrict__ a, const double *__restrict__ Kt,
                const double *__restrict__ s, int64_t nslots, uint16_t *A) {
    const int tk = blockIdx.x, ti = blockIdx.y;
    const int b = ti / (kBM / kGT), kc = tk / (kKC / kGT);
    if (kc > 2 * b + 1) return;
    extern __shared__ z_t gsm[];
    __shared__ z_t lt[kGT][kGT + 1];               // lt[r][c] = H(hi0 + r, lo0 + c)
    __shared__ z_t ui[kGT], uj[kGT];
    __shared__ double dEi[kGT];
    const int R = md.rank_x;
    z_t *sai = gsm, *saj = gsm + kGT * R;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int hi = max(ti, tk), lo = min(ti, tk);
    const int hi0 = hi * kGT, lo0 = lo * kGT;
    stage_tile(hi0, lo0, N, R, a, u, dE, sai, saj, ui, uj, dEi);
    __syncthreads();
    for (int c = ty; c < kGT; c += 8) {
        const int I = hi0 + tx, J = lo0 + c;
        z_t h = zmk(0.0, 0.0);
        if (!(hi == lo && tx < c) && I < N && J < N)
            h = bse_element(I, J, R, sai + tx, saj + c, kGT, ui[tx], uj[c], dEi[tx], Nk, nb, md.w0,
                            Kt);
        lt[tx][c] = h;
    }
    __syncthreads();
    if (hi == lo)                                  // the upper half of a diagonal tile
        for (int c = ty; c < kGT; c += 8)
            if (tx < c) lt[tx][c] = zconj(lt[c][tx]);
    __syncthreads();
    const int64_t slot = (int64_t)b * (b + 1) + kc;
    for (int r = ty; r < kGT; r += 8) {
        const int i = ti * kGT + r, k = tk * kGT + tx;   // row i, consecutive k
        z_t h = zmk(0.0, 0.0);
        if (i < N && k < N) {
            h = ti >= tk ? lt[r][tx] : zconj(lt[tx][r]);
            h = zscale(h, s[i] * s[k]);
        }
        const int row = i - b * kBM, col = k - kc * kKC;
        int tr[kS], tim[kS];
        split_digits(h.x, 0, tr);
        split_digits(h.y, 0, tim);
#pragma unroll
        for (int p = 0; p < kS; p++) {
            A[tri_index(2 * p, slot, nslots, row, col)] = bf16_exact(slice_value(tr[p], p));
            A[tri_index(2 * p + 1, slot, nslots, row, col)] = bf16_exact(slice_value(tim[p], p));
        }
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
    ChaseScalars *sc;
    int csplit;       // K chunks per split
    int tx, ty, tz;   // work units: column tiles x row tiles x splits
    unsigned long long *P;   // raw partials of the splits, layout below
    uint64_t wait_ns;        // limit of each bounded mbarrier wait
    int nslots;              // half storage: stored tiles per part, T (T + 1)
};

// One launch of the product kernel runs the work units of up to kMaxJobs
// independent products (a batch; one product alone is a batch of one).  Job
// j's units are numbered from unit0 on; each job keeps its own operands,
// tensor maps, K splits and partials, so its arithmetic is the same whatever
// else runs in the launch.
constexpr int kMaxJobs = 8;
struct OzJob {
    CUtensorMap tmA, tmB;    // slices of op(A) and of Y
    CUtensorMap tmA2;        // half storage: 64-row boxes of the stored tiles
    OzArgs args;
    int unit0;               // first unit of this job in the launch
};
struct OzBatch {
    OzJob job[kMaxJobs];
    int njobs;
    int units;               // units of all jobs
};

// Limit of each wait of the wind-down after an expired wait: long enough for
// any copy or MMA already issued to finish.
constexpr uint64_t kWindDownNs = 2000000000ull;

// Raw partial product of split z for output (i, j): per (z, j) three blocks
// of M 8-byte words, S of the real part (int64), S of the imaginary part
// (int64), and the FP32 tails T of both parts (float2), so that the splits
// are summed exactly in integers before the single FP64 recombination
// C = 2^(e_i + f_j) (S 2^-40 + T) in the reduction kernels.
constexpr int kPartWords = 3;
__host__ __device__ __forceinline__ int64_t part_word(int z, int n, int j, int blk, int64_t M, int64_t i) {
    return (((int64_t)z * n + j) * kPartWords + blk) * M + i;
}

// Exact diagonal g sums, per chunk, 2 kKC products (a Re and an Im MMA per
// K step) of each slice pair (p, g - p), in units of its own weight.  A digit
// of slice 1 is at most 2^8 in magnitude (|x| < 2^E, 48 bits: the leading
// digit carries the rounding), the others at most 2^7.  FP32 holds every
// integer up to 2^24 exactly, so the tensor core may sum drain_period(g)
// chunks before the drain warps move the accumulator into the 64-bit sums.
// The periods divide one another and the last diagonal (g = kEx) drains
// every chunk, last.
__host__ __device__ constexpr long long pair_bound(int p, int q) {
    return (long long)(p == 1 ? 256 : 128) * (q == 1 ? 256 : 128);
}
__host__ __device__ constexpr long long diag_bound(int g) {   // per chunk
    long long b = 0;
    for (int p = 1; p < g; p++) b += pair_bound(p, g - p);
    return 2 * kKC * b;
}
__host__ __device__ constexpr int drain_period(int g) { return g <= 3 ? 2 : 1; }
// The tail (diagonals above kEx) accumulates in FP32 over one work unit,
// and a unit spans at most kUnitChunks K chunks (the host splits K so).
// The tensor core's FP32 accumulation truncates: over a whole K of 50000 the
// tail's error grew to ~1e-11 of ||H|| ||y|| for eigenvector-like columns,
// enough to hold converged residuals near 5e-11 and cost 7 of 15 iterations
// at a tolerance of 1e-10 (N = 50000); over 2048 of K it is about 5e-12 and
// the solve takes the oracle's 8 iterations.
constexpr int kUnitChunks = 32;
static_assert(drain_period(2) * diag_bound(2) <= (1ll << 24) && drain_period(3) * diag_bound(3) <= (1ll << 24) &&
                  drain_period(4) * diag_bound(4) <= (1ll << 24) && drain_period(5) * diag_bound(5) <= (1ll << 24),
              "exact FP32 sums of the exact diagonals");
static_assert(drain_period(4) == 1 && drain_period(5) == 1, "the last two exact diagonals drain every chunk");

// Slice order q of the chunk's first pass (Re of slice p = 1), whose MMAs
// wait for their operands: the tail diagonals first (no drain), then g = 4
// and g = 5 (drained last in the previous chunk), then the B slices q = 2, 1
// (q = 2 is released last in the previous chunk, after pass (5, Im)).
template <int S>
struct FirstPassOrder {
    int q[S] = {};
    __host__ __device__ constexpr FirstPassOrder() {
        int n = 0;
        for (int t = S; t >= 5; t--) q[n++] = t;   // tail: g = 1 + t > 5
        q[n++] = 3;
        q[n++] = 4;
        q[n++] = 2;
        q[n++] = 1;
    }
};
// Diagonal g is drained after chunk cl (0-based within a unit of nc chunks).
__host__ __device__ __forceinline__ bool drain_due(int g, int cl, int nc) {
    return (cl + 1) % drain_period(g) == 0 || cl + 1 == nc;
}

// Issue order of the TMA producer within one K chunk.  Items: A slice p
// (its Re and Im tiles, read by passes 2(p-1) and 2(p-1) + 1, share one stage
// and one barrier pair) and B slice q.  Each load first waits for its buffer
// to be released by an earlier chunk; issuing the loads in the order of
// those releases (then of need) keeps one late release from holding back
// loads that could already go.  Positions are counted in slices p:
//   A slice p reuses the stage of slice p - kAPairs (released after its Im
//   pass).  B slice q >= 2 reuses its own buffer, last read in the previous
//   chunk by the Im pass of p = S + 1 - q; the slices q >= S - 2 are released
//   together after the Im pass of p = 3.  B slice 1 alternates between two
//   buffers; its buffer was last read by the final pass of the chunk before
//   the previous one.
// One barrier wait and one release per slice instead of per pass: every
// mbarrier operation the MMA thread issues between MMAs costs tensor issue
// time.
template <int S>
struct ProducerOrder {
    int kind[2 * S] = {};   // 0: A slice, 1: B slice
    int idx[2 * S] = {};    // slice p - 1, or slice q
    __host__ __device__ constexpr ProducerOrder() {
        int wt[2 * S] = {}, need[2 * S] = {};
        int n = 0;
        for (int pp = 0; pp < S; pp++, n++) {
            kind[n] = 0; idx[n] = pp; wt[n] = pp - kAPairs; need[n] = 8 * pp;
        }
        for (int q = 1; q <= S; q++, n++) {
            kind[n] = 1; idx[n] = q;
            wt[n] = (q == 1) ? -S - 1 : (q >= S - 2) ? 2 - S : -q;
            need[n] = S - q;
        }
        for (int i = 1; i < 2 * S; i++)       // insertion sort on (wait, need)
            for (int j = i; j > 0; j--) {
                const bool sw = wt[j] < wt[j - 1] ||
                                (wt[j] == wt[j - 1] && need[j] < need[j - 1]);
                if (!sw) break;
                int t = wt[j];
                wt[j] = wt[j - 1]; wt[j - 1] = t;
                t = need[j]; need[j] = need[j - 1]; need[j - 1] = t;
                t = kind[j]; kind[j] = kind[j - 1]; kind[j - 1] = t;
                t = idx[j]; idx[j] = idx[j - 1]; idx[j - 1] = t;
            }
    }
};

// A persistent kernel: one CTA per SM walks the work units u = blockIdx.x,
// blockIdx.x + gridDim.x, ... of a batch of products (usually one).  A unit
// is 128 rows x kW complex columns of one product's C over the K chunks of
// one split (at most kUnitChunks), numbered job by job, and within a job
// column tile fastest, then row tile, then split (so the CTAs running at one
// time share the operand slices of one K range in L2).  TMEM, the barriers
// and the pipelines live for the whole launch: the next unit's loads and MMAs
// start while the previous one drains, and no SM waits between CTAs.  Every
// role counts the chunks it has processed (gc) and the units' tails (ts), and
// all barrier phases follow from them.
//
// Per K chunk the MMA warp runs 2S passes, (p, Re H) then (p, Im H) for
// p = 1..S, and in each pass the slices q = S+1-p down to 1 of Y (the first
// pass in FirstPassOrder): accumulator of diagonal g = p + q gets
// Re H_p x [Yr | Yi]_q (Re pass) and Im H_p x [-Yi | Yr]_q (Im pass), four
// K=16 MMAs each.  Diagonal g's chunk sum starts at pair (1, g-1) and ends at
// pair (g-1, 1), so the exact accumulators that are due (drain_due) are
// drained in the order g = 2, 3, 4, 5 while later passes run.  The tail
// (g >= EXT+1) accumulates over the unit's chunks in its own columns: its
// weight is at most 2^-32 of the leading diagonal, so the tensor core's
// truncating FP32 sums there stay far below FP64 rounding of the result.
// The drain warps store S and the FP32 tail of each output raw; the
// reduction kernels sum the K splits and recombine.
template <class Cfg>
__global__ void __launch_bounds__(kThreads, 1)
k_ozaki_zgemm(const __grid_constant__ OzBatch bt) {
    constexpr int S = Cfg::kSl;
    constexpr int S2 = 2 * S;
    constexpr int kEx = Cfg::kEx;              // diagonals 2..kEx exact
    static_assert(kEx == 5 && S >= 4 && S <= 6,
                  "FirstPassOrder and the barrier groups assume kEx = 5 and 4 <= S <= 6");
    constexpr int kNEx = kEx - 1;              // exact accumulators
    constexpr bool kTail = Cfg::kTail;
    constexpr bool kTri = Cfg::kTri;
    constexpr int kNB = S + 1;                 // B buffers: slices 1..S, slice 1 twice
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;                                        // kAPairs x (Re, Im) x 16 KB
    uint8_t *sB = sm + kAStages * kATile;                    // kNB x [-Yi | Yr | Yi]
    // fullB[0][gc & 1]: B slices q >= 3 of chunk gc have landed (S - 2
    // arrivals), fullB[1][gc & 1]: slices 2 and 1.  The two barriers of a group
    // alternate so that slice 1 of the next chunk, whose buffer frees early,
    // never arrives on the phase of the current one.
    // emptyB[b]: B buffer b may be refilled; the buffers of slices q >= S - 2
    // (last read by the Im passes of p = 1, 2, 3) share emptyBg instead, one
    // release after p = 3
    __shared__ uint64_t fullA[kAPairs], emptyA[kAPairs], fullB[2][2], emptyB[kNB], emptyBg;
    // accEmpty[0]: the exact accumulators g <= kEx - 1 of the chunk have been
    // read, accEmpty[1]: g = kEx too (the drain warps read them in the order
    // g = 2, ..., kEx)
    __shared__ uint64_t accFull[kNEx], accEmpty[2], tailFull, tailEmpty;
    // mmaDone: the wind-down commit of the MMA thread (every MMA it issued
    // has completed)
    __shared__ uint64_t mmaDone;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int units = bt.units;
    const uint64_t wait_ns = bt.job[0].args.wait_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAPairs; s++) { tc::mbar_init(&fullA[s], 1); tc::mbar_init(&emptyA[s], 1); }
        for (int s = 0; s < kNB; s++) tc::mbar_init(&emptyB[s], 1);
        tc::mbar_init(&emptyBg, 1);
        for (int s = 0; s < 2; s++) {
            tc::mbar_init(&fullB[0][s], S - 2);
            tc::mbar_init(&fullB[1][s], 2);
        }
        for (int s = 0; s < kNEx; s++) tc::mbar_init(&accFull[s], 1);
        tc::mbar_init(&accEmpty[0], kDrainWarps);
        tc::mbar_init(&accEmpty[1], kDrainWarps);
        tc::mbar_init(&tailFull, 1);
        tc::mbar_init(&tailEmpty, kDrainWarps);
        tc::mbar_init(&mmaDone, 1);
        abort_flag = 0;
        tc::mbar_fence_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_base, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;

    // B buffer of slice q in chunk gc of this CTA, and how many times that
    // buffer was filled before
    auto bbuf = [](int q, int gc) { return q == 1 ? ((gc & 1) ? S : 0) : q - 1; };
    auto buse = [](int q, int gc) { return q == 1 ? (gc >> 1) : gc; };
    // unit -> job, column tile, row tile, K range
    auto unit = [&](int u, int &jb, int &j0, int64_t &i0, int &z, int &c0, int &c1) {
        jb = 0;
        while (jb + 1 < bt.njobs && u >= bt.job[jb + 1].unit0) jb++;
        const OzArgs &a = bt.job[jb].args;
        const int ul = u - bt.job[jb].unit0;
        const int x = ul % a.tx, y = (ul / a.tx) % a.ty;
        z = ul / (a.tx * a.ty);
        j0 = x * kW;
        i0 = (int64_t)y * kBM;
        c0 = z * a.csplit;
        c1 = min(a.nchunks, c0 + a.csplit);
    };

    // Where the producer stopped: chunk ab_gc, item ab_it of ProducerOrder
    // (items before it issued).  The wind-down after an expired wait derives
    // from these which phases of the full barriers were armed.
    int ab_gc = 0, ab_it = 0;
    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            for (int j = 0; j < bt.njobs; j++) {
                tc::prefetch_tmap(&bt.job[j].tmA);
                tc::prefetch_tmap(&bt.job[j].tmB);
                if (kTri) tc::prefetch_tmap(&bt.job[j].tmA2);
            }
            constexpr ProducerOrder<S> order;
            bool ok = true;
            int gc = 0;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                int jb, j0, z, c0, c1;
                int64_t i0;
                unit(u, jb, j0, i0, z, c0, c1);
                const CUtensorMap *tmA = &bt.job[jb].tmA, *tmB = &bt.job[jb].tmB;
                const CUtensorMap *tmA2 = &bt.job[jb].tmA2;
                const int nch = bt.job[jb].args.nchunks, ns = bt.job[jb].args.nslots;
                const int br = (int)(i0 / kBM);           // row tile
                for (int c = c0; c < c1 && ok; c++, gc++) {
                    ab_gc = gc;
                    // half storage: chunk c lies above the stored triangle of
                    // row tile br, so its A tile is read from the stored tiles
                    // (c / 2, 2 br) and (c / 2, 2 br + 1), rows 64 (c % 2) on
                    const bool mir = kTri && c > 2 * br + 1;
#pragma unroll
                    for (int it = 0; it < 2 * S; it++) {
                        if (order.kind[it] == 0) {
                            const int pp = order.idx[it];
                            const int ua = S * gc + pp, st = ua % kAPairs, n = ua / kAPairs;
                            if (n >= 1 && !tc::mbar_wait(&emptyA[st], (n - 1) & 1, &abort_flag, wait_ns)) {
                                ok = false;
                                ab_it = it;
                                break;
                            }
                            tc::mbar_expect_tx(&fullA[st], 2 * kATile);
                            // parts (slice p, re) and (slice p, im) = 2 pp, 2 pp + 1 in the
                            // A tensor's part order
                            uint8_t *adst = sA + st * 2 * kATile;
                            if (!kTri) {
                                tc::tma_load_3d(adst, tmA, 0, (int)i0, (2 * pp) * nch + c, &fullA[st]);
                                tc::tma_load_3d(adst + kATile, tmA, 0, (int)i0, (2 * pp + 1) * nch + c, &fullA[st]);
                            } else if (!mir) {
                                const int zt = br * (br + 1) + c;            // stored tile (br, c)
                                tc::tma_load_3d(adst, tmA, 0, 0, (2 * pp) * ns + zt, &fullA[st]);
                                tc::tma_load_3d(adst + kATile, tmA, 0, 0, (2 * pp + 1) * ns + zt, &fullA[st]);
                            } else {
                                const int bc = c >> 1, zt = bc * (bc + 1) + 2 * br, y = (c & 1) * 64;
#pragma unroll
                                for (int r = 0; r < 2; r++) {
                                    uint8_t *d = adst + r * kATile;
                                    tc::tma_load_3d(d, tmA2, 0, y, (2 * pp + r) * ns + zt, &fullA[st]);
                                    tc::tma_load_3d(d + kATile / 2, tmA2, 0, y, (2 * pp + r) * ns + zt + 1, &fullA[st]);
                                }
                            }
                        } else {
                            const int q = order.idx[it];
                            const int b = bbuf(q, gc), n = buse(q, gc);
                            if (n >= 1 && !tc::mbar_wait(q >= S - 2 ? &emptyBg : &emptyB[b], (n - 1) & 1, &abort_flag, wait_ns)) {
                                ok = false;
                                ab_it = it;
                                break;
                            }
                            uint64_t *fb = &fullB[q >= 3 ? 0 : 1][gc & 1];
                            tc::mbar_expect_tx(fb, kBSlice);
                            uint8_t *bdst = sB + b * kBSlice;
                            // smem [-Yi | Yr | Yi] from parts 2, 0, 1
                            tc::tma_load_3d(bdst + 0 * kBPart, tmB, 0, j0, ((q - 1) * 3 + 2) * nch + c, fb);
                            tc::tma_load_3d(bdst + 1 * kBPart, tmB, 0, j0, ((q - 1) * 3 + 0) * nch + c, fb);
                            tc::tma_load_3d(bdst + 2 * kBPart, tmB, 0, j0, ((q - 1) * 3 + 1) * nch + c, fb);
                        }
                    }
                }
            }
            if (ok) {
                ab_gc = gc;      // every chunk issued in full
                ab_it = 0;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, kN);
            // descriptors of the first A stage and B buffer; the others are
            // offsets in 16-byte units of the 14-bit address field (the whole
            // operand area lies below 256 KB, so no carry leaves the field)
            const uint64_t adesc0 = tc::sdesc_sw128(sA), bdesc0 = tc::sdesc_sw128(sB);
            // half storage, chunks above the stored triangle: the two 64-row
            // halves of each A tile read MN-major (transposed), the Im pass
            // negated (the tile is conj(H) transposed)
            const uint64_t adescT0 = tc::sdesc_sw128_mn(sA, kATile / 2);
            constexpr uint32_t idescT = idesc | tc::kIdescTransA;
            constexpr uint32_t idescTN = idescT | tc::kIdescNegA;
            constexpr FirstPassOrder<S> kFirst;
            bool ok = true;
            int gc = 0, uc = 0, ts = 0;   // ts: unit tails committed
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x, uc++) {
                int jb, j0, z, c0, c1;
                int64_t i0;
                unit(u, jb, j0, i0, z, c0, c1);
                const int br = (int)(i0 / kBM);
                for (int c = c0; c < c1 && ok; c++, gc++) {
                    const int cl = c - c0, nc = c1 - c0;
                    const bool first = cl == 0;   // the unit's first chunk
                    const bool mir = kTri && c > 2 * br + 1;
#pragma unroll
                    for (int pi = 0; pi < S2; pi++) {
                        const int p = pi / 2 + 1, ri = pi & 1;
                        const int ua = S * gc + (p - 1), st = ua % kAPairs;
                        if (ri == 0) {
                            if (!tc::mbar_wait(&fullA[st], (ua / kAPairs) & 1, &abort_flag, wait_ns)) { ok = false; break; }
                            tc::fence_after();
                        }
                        const uint64_t a0 = (mir ? adescT0 : adesc0) + (uint64_t)((st * 2 * kATile + ri * kATile) >> 4);
                        // K step of 16: 32 bytes along a K-major row, 16 rows of
                        // 128 bytes MN-major
                        const uint32_t ak = mir ? 128u : 2u;
                        const uint32_t id = !mir ? idesc : (ri == 0 ? idescT : idescTN);
                        // One MMA: K step kk of slice pair (p, q).
                        // coll: the A-collector use of the first pass (0: none)
                        auto step = [&](int kk, int q, int coll) -> bool {
                            const int g = p + q;
                            const int b = bbuf(q, gc);
                            if (pi == 0 && kk == 0) {
                                // B slices before the first MMA of their group (the
                                // chunk's first MMA reads slice FirstPassOrder.q[0] >= 3)
                                if ((q == kFirst.q[0] || q == 2) &&
                                    !tc::mbar_wait(&fullB[q >= 3 ? 0 : 1][gc & 1], (gc >> 1) & 1, &abort_flag, wait_ns))
                                    return false;
                                // the previous chunk's accumulators g <= kEx - 1 before
                                // the first of them (g = kEx - 1, q = 3), g = kEx at q = 4
                                if ((g == kEx - 1 || g == kEx) && gc >= 1 &&
                                    !tc::mbar_wait(&accEmpty[g == kEx ? 1 : 0], (gc - 1) & 1, &abort_flag, wait_ns))
                                    return false;
                                // the tail of the previous unit must have been read
                                if (g > kEx && first && q == S && ts >= 1 &&
                                    !tc::mbar_wait(&tailEmpty, (ts - 1) & 1, &abort_flag, wait_ns)) return false;
                                tc::fence_after();
                            }
                            const uint32_t d = tmem + (uint32_t)((g <= kEx ? g - 2 : kNEx) * kN);
                            // Re pass: [Yr | Yi] (parts 1, 2); Im pass: [-Yi | Yr] (parts 0, 1)
                            const uint64_t b0 =
                                bdesc0 + (uint64_t)((b * kBSlice + (ri == 0 ? kBPart : 0)) >> 4);
                            // a fresh sum: every exact diagonal at its first pair
                            // of the chunk, the tail at its first pair of the unit
                            const bool fresh = (g <= kEx) ? (pi == 0 && q == g - 1 && cl % drain_period(g) == 0)
                                                          : (first && pi == 0 && q == S);
                            const uint32_t acc = (fresh && kk == 0) ? 0u : 1u;
                            const uint64_t a = a0 + ak * kk, bd = b0 + 2 * kk;
                            if (pi == 0 && coll == tc::A_FILL)
                                tc::mma_bf16_ca<tc::A_FILL>(d, a, bd, id, acc);
                            else if (pi == 0 && coll == tc::A_LASTUSE)
                                tc::mma_bf16_ca<tc::A_LASTUSE>(d, a, bd, id, acc);
                            else if (pi == 0 || p == S)
                                tc::mma_bf16(d, a, bd, id, acc);
                            else if (q == S + 1 - p)
                                tc::mma_bf16_ca<tc::A_FILL>(d, a, bd, id, acc);
                            else if (q == 1)
                                tc::mma_bf16_ca<tc::A_LASTUSE>(d, a, bd, id, acc);
                            else
                                tc::mma_bf16_ca<tc::A_USE>(d, a, bd, id, acc);
                            return true;
                        };
                        if (pi == 0) {
                            // the chunk's first pass in FirstPassOrder, two slices at a
                            // time, so the operands released last in the previous
                            // chunk are needed last; the two MMAs of one K step share
                            // A through the collector buffer (an odd S ends with
                            // one slice, A read from shared memory)
#pragma unroll
                            for (int t = 0; t < S; t += 2) {
                                const int qa = kFirst.q[t];
                                if (t + 1 == S) {
                                    if (!step(0, qa, 0)) {
                                        ok = false;
                                        break;
                                    }
#pragma unroll
                                    for (int kk = 1; kk < kKC / 16; kk++) step(kk, qa, 0);
                                    continue;
                                }
                                const int qb = kFirst.q[t + 1 < S ? t + 1 : 0];
                                if (!step(0, qa, tc::A_FILL) || !step(0, qb, tc::A_LASTUSE)) {
                                    ok = false;   // fails only in a wait
                                    break;
                                }
#pragma unroll
                                for (int kk = 1; kk < kKC / 16; kk++) {
                                    step(kk, qa, tc::A_FILL);
                                    step(kk, qb, tc::A_LASTUSE);
                                }
                            }
                        } else {
                            // kk outer, q inner: the MMAs of one K step share their A
                            // tile, read from shared memory once into the collector
                            // buffer and reused for every slice q of Y (not for a
                            // single pair)
#pragma unroll
                            for (int kk = 0; kk < kKC / 16; kk++) {
#pragma unroll
                                for (int q = S + 1 - p; q >= 1; q--) step(kk, q, 0);   // no waits
                            }
                        }
                        if (!ok) break;
                        if (ri == 1) {
                            tc::mma_commit(&emptyA[st]);
                            // last reader of B slice S + 1 - p; last pair of diagonal p + 1
                            const int qd = S + 1 - p;
                            if (qd < S - 2) tc::mma_commit(&emptyB[bbuf(qd, gc)]);
                            else if (p == 3) tc::mma_commit(&emptyBg);
                            if (p + 1 <= kEx && drain_due(p + 1, cl, nc)) tc::mma_commit(&accFull[p - 1]);
                        }
                    }
                    // the chunk's last MMA is a tail pair (p = S, q = 1)
                    if (ok && kTail && cl + 1 == nc) {
                        tc::mma_commit(&tailFull);
                        ts++;
                    }
                }
            }
        }
    } else {
        // ------------------------------------------------ drain + epilogue
        // warp w: TMEM lanes of quadrant (w & 3); columns [half*kW, half*kW+kW)
        // of every accumulator (half 0: re, half 1: im).
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        bool ok = true;
        int gc = 0, ts = 0;                        // ts: unit tails read
        int dn[kNEx] = {};                         // drains of each exact diagonal so far
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            int jb, j0, z, c0, c1;
            int64_t i0;
            unit(u, jb, j0, i0, z, c0, c1);
            const OzArgs &args = bt.job[jb].args;
            long long Sx[kHalf];
#pragma unroll
            for (int j = 0; j < kHalf; j++) Sx[j] = 0;
            // the unit's outputs: row i, columns j0 + v < n; the FP32 tail goes
            // to the raw partials straight from TMEM (registers are full)
            const int jn = args.n - j0;
            const int64_t i = i0 + row;
            float *Pt = (float *)args.P;
            for (int c = c0; c < c1 && ok; c++, gc++) {
#pragma unroll 1
                for (int g = 2; g <= kEx; g++) {
                    if (!drain_due(g, c - c0, c1 - c0)) continue;
                    if (!tc::mbar_wait(&accFull[g - 2], dn[g - 2] & 1, &abort_flag, wait_ns)) { ok = false; break; }
                    dn[g - 2]++;
                    tc::fence_after();
                    const uint32_t col = (uint32_t)((g - 2) * kN + half * kHalf);
                    const float scale = __int_as_float((127 + kBeta * g) << 23);   // 2^(8g)
                    const int shift = kBeta * (5 - g);                             // S in units of 2^-40
                    // 16 columns at a time (registers are the limit here)
#pragma unroll
                    for (int h = 0; h < kHalf; h += 16) {
                        uint32_t r[16];
                        tc::tmem_ld16(tmem + lane_addr + col + h, r);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int v = 0; v < 16; v++) {
                            const int dv = __float2int_rn(__uint_as_float(r[v]) * scale);
                            Sx[h + v] += (long long)dv << shift;
                        }
                    }
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0 && g >= kEx - 1) tc::mbar_arrive(&accEmpty[g == kEx ? 1 : 0]);
                }
                if (ok && kTail && c + 1 == c1) {
                    if (!tc::mbar_wait(&tailFull, ts & 1, &abort_flag, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t col = (uint32_t)(kNEx * kN + half * kHalf);
                    // tail slot of column j0 + v: tb + v * (2 * kPartWords * M) floats
                    float *tb = Pt + 2 * part_word(z, args.n, j0, 2, args.M, i) + half;
                    const int64_t tstep = 2 * kPartWords * args.M;
#pragma unroll 1
                    for (int h = 0; h < kHalf; h += 8) {
                        uint32_t r[8];
                        tc::tmem_ld8(tmem + lane_addr + col + h, r);
                        tc::tmem_wait_ld();
                        if (i < args.M) {
#pragma unroll
                            for (int v = 0; v < 8; v++) {
                                if (h + v >= jn) break;
                                tb[(h + v) * tstep] = __uint_as_float(r[v]);
                            }
                        }
                    }
                    ts++;
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tailEmpty);
                }
            }
            if (!ok) break;
            // Raw partials of this split: S (int64) beside the FP32 tail; the
            // reduction kernels sum the splits exactly and recombine once.
            if (i < args.M) {
                unsigned long long *P = args.P;
#pragma unroll
                for (int v = 0; v < kHalf; v++) {
                    if (v >= jn) break;
                    P[part_word(z, args.n, j0 + v, half, args.M, i)] = (unsigned long long)Sx[v];
                    if (!kTail) Pt[2 * part_word(z, args.n, j0 + v, 2, args.M, i) + half] = 0.f;
                }
            }
        }
    }

    tc::fence_before();
    __syncthreads();
    if (abort_flag) {
        // Wind-down after an expired wait: every role has left its loop, so
        // no new copy or MMA is issued.  Before the shared memory and TMEM are
        // released, the copies and MMAs already issued must finish:
        //  - producer: a B phase armed by only some of its slices gets its
        //    missing arrivals (the phase then completes once the bytes of
        //    the armed slices land), then every armed phase of every full
        //    barrier is waited for;
        //  - MMA thread: one more commit, which arrives once every MMA it
        //    issued has completed.
        bool drained = true;
        if (warp == 0 && lane == 0) {
            constexpr ProducerOrder<S> order;
            constexpr int kArr[2] = {S - 2, 2};
            // B: chunks before ab_gc armed both groups of their barrier in
            // full; chunk ab_gc armed the items before ab_it
            for (int g = 0; g < 2; g++) {
                int part = 0;
                for (int it = 0; it < ab_it; it++)
                    if (order.kind[it] == 1 && (order.idx[it] >= 3 ? 0 : 1) == g) part++;
                for (int par = 0; par < 2; par++) {
                    int ph = ab_gc / 2 + ((ab_gc & 1) && par == 0 ? 1 : 0);   // full chunks of parity par
                    if (par == (ab_gc & 1) && part > 0) {
                        for (int k = part; k < kArr[g]; k++) tc::mbar_arrive(&fullB[g][par]);
                        ph++;
                    }
                    if (ph > 0) drained &= tc::mbar_wait_for(&fullB[g][par], (ph - 1) & 1, kWindDownNs);
                }
            }
            // A: the last fill of each stage, ua = S gc + pp
            for (int st = 0; st < kAPairs; st++) {
                int last = -1;
                for (int it = 0; it < ab_it; it++)
                    if (order.kind[it] == 0 && (S * ab_gc + order.idx[it]) % kAPairs == st)
                        last = max(last, S * ab_gc + order.idx[it]);
                if (last < 0 && S * ab_gc > 0) {
                    const int top = S * ab_gc - 1;
                    last = top - (((top - st) % kAPairs) + kAPairs) % kAPairs;
                }
                if (last >= 0) drained &= tc::mbar_wait_for(&fullA[st], (last / kAPairs) & 1, kWindDownNs);
            }
        }
        if (warp == 1 && lane == 0) {
            tc::mma_commit(&mmaDone);
            drained &= tc::mbar_wait_for(&mmaDone, 0, kWindDownNs);
        }
        if (!drained)
            for (int j = 0; j < bt.njobs; j++) set_error(bt.job[j].args.sc, DEV_TIMEOUT, -1 - (int)blockIdx.x);
        tc::fence_before();
        __syncthreads();
        if (threadIdx.x == 0)
            for (int j = 0; j < bt.njobs; j++) set_error(bt.job[j].args.sc, DEV_TIMEOUT, blockIdx.x);
    }
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// One output of the emulated product: the splits' S summed in int64 (exact)
// and T in FP32 (the tail is below 2^-32 of the result's scale), then
// C = 2^x (S 2^-40 + T), x = e_i + f_j.  The powers of two are built from
// exponent bits (FP64 issue is slow on this part).
__device__ __forceinline__ z_t recombine(const unsigned long long *__restrict__ P, int nsplit, int n,
                                         int j, int64_t M, int64_t i, int x) {
    long long sr = 0, si = 0;
    float tr = 0.f, ti = 0.f;
    for (int z = 0; z < nsplit; z++) {
        sr += (long long)P[part_word(z, n, j, 0, M, i)];
        si += (long long)P[part_word(z, n, j, 1, M, i)];
        const float2 t = ((const float2 *)P)[part_word(z, n, j, 2, M, i)];
        tr += t.x;
        ti += t.y;
    }
    if (x > -960 && x < 1000) {
        const double sc = __longlong_as_double((long long)(1023 + x) << 52);
        const double sc40 = __longlong_as_double((long long)(1023 - 40 + x) << 52);
        return zmk(fma((double)sr, sc40, (double)tr * sc), fma((double)si, sc40, (double)ti * sc));
    }
    return zmk(ldexp((double)sr * 0x1.0p-40 + (double)tr, x), ldexp((double)si * 0x1.0p-40 + (double)ti, x));
}

__device__ __forceinline__ int exp_or_zero(int e) { return e == INT_MIN ? 0 : e; }

// C = epi(H Y) from the splits' partials (summed in increasing z: deterministic).
// With ts (half storage): row i of the recombined product scaled by ts[i].
__global__ void k_split_reduce(int64_t M, int n, int nsplit, const unsigned long long *__restrict__ P,
                               const int *__restrict__ E, const int *__restrict__ F, GemmEpi ep,
                               const z_t *__restrict__ Y, int64_t ldy, z_t *C, int64_t ldc,
                               const double *__restrict__ ts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= M) return;
    z_t v = recombine(P, nsplit, n, j, M, i, exp_or_zero(E[i]) + exp_or_zero(F[j]));
    if (ts) v = zscale(v, ts[i]);
    if (ep.mode == GEMM_CHEB) {
        v = zscale(zsub(v, zscale(Y[i + j * ldy], ep.c)), ep.s1);
        if (ep.Yp) v = zsub(v, zscale(ep.Yp[i + j * ep.ldyp], ep.s2));
    }
    C[i + j * ldc] = v;
}

// General products: C = out(op(A) B) from the splits' partials.
// OZ_PLAIN: C = S; OZ_SUB: C = D - S (D may alias C); OZ_GRAM (square):
// C = S, or its Hermitian part (S + S^H)/2, plus shift on the diagonal.
__global__ void k_gen_reduce(int64_t M, int n, int nsplit, const unsigned long long *__restrict__ P,
                             const int *__restrict__ E, const int *__restrict__ F, int mode,
                             const z_t *D, int64_t ldd, double shift, int hermitize, z_t *C,
                             int64_t ldc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= M) return;
    z_t v = recombine(P, nsplit, n, j, M, i, exp_or_zero(E[i]) + exp_or_zero(F[j]));
    if (mode == OZ_SUB) {
        v = zsub(D[i + j * ldd], v);
    } else if (mode == OZ_GRAM) {
        if (hermitize) {
            const z_t t = recombine(P, nsplit, n, (int)i, M, j, exp_or_zero(E[j]) + exp_or_zero(F[i]));
            v = zmk(0.5 * (v.x + t.x), 0.5 * (v.y - t.y));
            if (i == j) v.y = 0.0;
        }
        if (i == j) v.x += shift;
    }
    C[i + j * ldc] = v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled of the CUDA driver API, looked up once (a thread-safe static).
EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (EncodeTiledFn)p;
        cudaGetLastError();
        return (EncodeTiledFn) nullptr;
    }();
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

// Split K into `sp` ranges so that the units (tiles x splits) spread
// evenly over one persistent CTA per SM.  Cost in K-chunk units: the
// busiest CTA's units, each with half a chunk of pipeline fill and drain,
// plus the raw partials written and summed by the reduction (48 bytes per
// complex output and split, at about one chunk per 6 us and 6 TB/s).  At
// least 16 K chunks per split, partials within the workspace; 0 if even one
// split does not fit.
// K splits of a product: at least enough that no work unit spans more than
// kUnitChunks K chunks (accuracy of the FP32 tail), then the count that
// spreads the units best over the SMs, within the partials' memory.
int choose_splits(int tiles, int nchunks, int n, int64_t M, size_t partial_bytes, int sms) {
    constexpr int64_t kPB = kPartWords * 8;       // bytes per complex output and split
    if ((int64_t)n * M * kPB > (int64_t)partial_bytes) return 0;
    const int sp0 = (nchunks + kUnitChunks - 1) / kUnitChunks;
    if ((int64_t)sp0 * n * M * kPB > (int64_t)partial_bytes) return 0;
    int best = sp0;
    double best_t = 1e30;
    for (int sp = sp0; sp <= sp0 + 32; sp++) {
        if ((int64_t)sp * 16 > nchunks && sp > sp0) break;
        if ((int64_t)sp * n * M * kPB > (int64_t)partial_bytes) break;
        const int64_t u = (int64_t)tiles * sp;
        const int64_t per = (u + sms - 1) / sms;
        const double chunks = (double)((nchunks + sp - 1) / sp);
        const double part = (double)sp * n * M * (2.0 * kPB) / (6.0e12 * 6.0e-6);
        const double t = (double)per * (chunks + 0.5) + part;
        if (t < best_t - 1e-9) { best_t = t; best = sp; }
    }
    return best;
}

}  // namespace

int64_t ozaki_padded(int64_t N) { return (N + 127) / 128 * 128; }

size_t ozaki_a_bytes(int64_t N) {
    const int64_t Np = ozaki_padded(N);
    return (size_t)kS * 2 * Np * Np * 2;
}

size_t ozaki_a_bytes_tri(int64_t N) {
    const int64_t T = ozaki_padded(N) / kBM;
    return (size_t)kS * 2 * T * (T + 1) * kBM * kKC * 2;
}

size_t ozaki_partial_bytes(int64_t N, int m) {
    const int mp = (m + kW - 1) / kW * kW;
    // splits x columns: the minimum split count of a product with K = N at
    // full width, or 8 splits, or 16 tiles' worth for narrow products
    const int64_t nch = ozaki_padded(N) / kKC;
    const int64_t sp0 = (nch + kUnitChunks - 1) / kUnitChunks;
    return (size_t)N * (kPartWords * 8) *
           std::max<int64_t>(16 * kW, std::max<int64_t>(8, sp0) * (int64_t)mp);
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
    oh->tri = false;
    k_fill_int<<<(unsigned)((Np + 255) / 256), 256, 0, st>>>(oh->E, (int)Np, INT_MIN);
    bse_count_launches(1);
    const int cpb = 256;
    dim3 g1((unsigned)((N + 255) / 256), (unsigned)((N + cpb - 1) / cpb));
    k_row_exponent<<<g1, 256, 0, st>>>(N, N, H, ldh, oh->E, cpb, sc);
    bse_count_launches(1);
    dim3 g2((unsigned)(Np / 32), (unsigned)(Np / 32));
    k_slice_h<<<g2, dim3(32, 8), 0, st>>>(N, Np, N, Np, H, ldh, oh->E, (uint16_t *)oh->A);
    bse_count_launches(1);
    if (!make_map((CUtensorMap *)oh->tmap, oh->A, (uint64_t)Np, (uint64_t)(kS * 2 * (Np / kKC)),
                  kBM))
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t ozaki_prepare_h_tri(int64_t N, const z_t *H, int64_t ldh, OzakiH *oh,
                                ChaseScalars *sc, cudaStream_t st) {
    const int64_t Np = ozaki_padded(N), T = Np / kBM, nslots = T * (T + 1);
    oh->N = N;
    oh->Np = Np;
    oh->tri = true;
    unsigned long long *Mx = (unsigned long long *)oh->s;
    cudaError_t e = cudaMemsetAsync(Mx, 0, (size_t)Np * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const unsigned Tt = (unsigned)((N + 31) / 32), Tp = (unsigned)(Np / 32);
    k_tri_rowmax<<<dim3(Tt, Tt), dim3(32, 8), 0, st>>>(N, H, ldh, Mx);
    k_tri_scales<<<(unsigned)((Np + 255) / 256), 256, 0, st>>>(N, Np, Mx, oh->t, oh->s, oh->E, sc);
    k_slice_tri<<<dim3(Tp, Tp), dim3(32, 8), 0, st>>>(N, H, ldh, oh->s, nslots, (uint16_t *)oh->A);
    bse_count_launches(3);
    if (!make_map((CUtensorMap *)oh->tmap, oh->A, kBM, (uint64_t)(kS * 2 * nslots), kBM) ||
        !make_map((CUtensorMap *)oh->tmap2, oh->A, kBM, (uint64_t)(kS * 2 * nslots), kBM / 2))
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t ozaki_prepare_bse(int Nk, int Nv, int Nc, const BseModel &md, const double *dE,
                              const z_t *u, const z_t *a, const double *Kt, bool tri, OzakiH *oh,
                              ChaseScalars *sc, cudaStream_t st) {
    const int64_t N = (int64_t)Nk * Nv * Nc;
    const int64_t Np = ozaki_padded(N), Tb = Np / kBM, nslots = Tb * (Tb + 1);
    oh->N = N;
    oh->Np = Np;
    oh->tri = tri;
    const int dyn = 2 * kGT * std::max(md.rank_x, 1) * (int)sizeof(z_t);
    static std::once_flag once[3][kMaxDevices];
    static cudaError_t attr[3][kMaxDevices];
    cudaError_t ae = smem_attr_once(once[0], attr[0], (const void *)k_gen_row_exponent, 2 * kGT * 64 * (int)sizeof(z_t));
    if (ae == cudaSuccess)
        ae = smem_attr_once(once[1], attr[1], (const void *)k_gen_slice, 2 * kGT * 64 * (int)sizeof(z_t));
    if (ae == cudaSuccess)
        ae = smem_attr_once(once[2], attr[2], (const void *)k_gen_slice_tri, 2 * kGT * 64 * (int)sizeof(z_t));
    if (ae != cudaSuccess) return ae;
    const unsigned T = (unsigned)((N + kGT - 1) / kGT), Tp = (unsigned)(Np / kGT);
    if (tri) {
        unsigned long long *Mx = (unsigned long long *)oh->s;
        ae = cudaMemsetAsync(Mx, 0, (size_t)Np * sizeof(unsigned long long), st);
        if (ae != cudaSuccess) return ae;
        k_gen_row_exponent<<<dim3(T, T), dim3(kGT, 8), dyn, st>>>(Nk, Nv * Nc, (int)N, md, dE, u, a,
                                                                  Kt, oh->E, sc, Mx);
        k_tri_scales<<<(unsigned)((Np + 255) / 256), 256, 0, st>>>(N, Np, Mx, oh->t, oh->s, oh->E, sc);
        k_gen_slice_tri<<<dim3(Tp, Tp), dim3(kGT, 8), dyn, st>>>(Nk, Nv * Nc, (int)N, md, dE, u, a,
                                                                 Kt, oh->s, nslots,
                                                                 (uint16_t *)oh->A);
        bse_count_launches(3);
        if (!make_map((CUtensorMap *)oh->tmap, oh->A, kBM, (uint64_t)(kS * 2 * nslots), kBM) ||
            !make_map((CUtensorMap *)oh->tmap2, oh->A, kBM, (uint64_t)(kS * 2 * nslots), kBM / 2))
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    k_fill_int<<<(unsigned)((Np + 255) / 256), 256, 0, st>>>(oh->E, (int)Np, INT_MIN);
    bse_count_launches(1);
    k_gen_row_exponent<<<dim3(T, T), dim3(kGT, 8), dyn, st>>>(Nk, Nv * Nc, (int)N, md, dE, u, a, Kt,
                                                              oh->E, sc, nullptr);
    k_gen_slice<<<dim3(Tp, Tp), dim3(kGT, 8), dyn, st>>>(Nk, Nv * Nc, (int)N, Np, md, dE, u, a, Kt,
                                                        oh->E, (uint16_t *)oh->A);
    bse_count_launches(2);
    if (!make_map((CUtensorMap *)oh->tmap, oh->A, (uint64_t)Np, (uint64_t)(kS * 2 * (Np / kKC)),
                  kBM))
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

namespace {

template <class Cfg>
cudaError_t launch_variant(const OzBatch &b, int sms, cudaStream_t st) {
    static std::once_flag once[kMaxDevices];
    static cudaError_t attr[kMaxDevices];
    {
        const cudaError_t ae = smem_attr_once(once, attr, (const void *)k_ozaki_zgemm<Cfg>, Cfg::kSmem);
        if (ae != cudaSuccess) return ae;
    }
    const dim3 grid((unsigned)std::min(b.units, sms));
    k_ozaki_zgemm<Cfg><<<grid, kThreads, Cfg::kSmem, st>>>(b);
    bse_count_launches(1);
    return cudaGetLastError();
}

// Kernel configuration of a launch: the accuracy level (OzLevel), plus
// kOzTri for half storage.
constexpr int kOzTri = 4;
cudaError_t launch_batch(const OzBatch &b, int cfg, int sms, cudaStream_t st) {
    switch (cfg) {
    case OZ_S4: return launch_variant<CfgMixed>(b, sms, st);
    case OZ_S5: return launch_variant<CfgMid>(b, sms, st);
    case OZ_S6 | kOzTri: return launch_variant<CfgFP64Tri>(b, sms, st);
    case OZ_S4 | kOzTri: return launch_variant<CfgMixedTri>(b, sms, st);
    case OZ_S5 | kOzTri: return launch_variant<CfgMidTri>(b, sms, st);
    default: return launch_variant<CfgFP64>(b, sms, st);
    }
}

// A batch of one product.
OzBatch single(const CUtensorMap &tmA, const CUtensorMap &tmB, const OzArgs &a) {
    OzBatch b;
    memset(&b, 0, sizeof b);
    b.job[0].tmA = tmA;
    b.job[0].tmB = tmB;
    b.job[0].args = a;
    b.job[0].unit0 = 0;
    b.njobs = 1;
    b.units = a.tx * a.ty * a.tz;
    return b;
}

}  // namespace

// ------------------------------------------------------ product batcher
// Products that solver threads of one process submit at about the same time
// run in one launch of the kernel.  A submitting thread records an event on
// its stream (its operand slices are ready) and queues its job; the first
// queued thread leads: it waits until as many jobs are queued as there are
// active solvers (each of them is then waiting on a product) or until the
// window has passed since it began to lead, then launches every queued job
// of the same kernel configuration (up to kMaxJobs, oldest first) on the batcher's
// stream behind the jobs' events, records one event after the launch, and
// hands the lead on.  Every submitter makes its stream wait for that event
// before its split reduction.  The jobs' units, splits and operands are
// those of the product alone, so results are the same, bit for bit.
struct OzBatcher {
    std::mutex mu;
    std::condition_variable cv;
    struct Pending {
        OzJob job;
        int cfg = OZ_S6;         // kernel configuration (launch_batch)
        cudaEvent_t ready = nullptr, done = nullptr;
        bool launched = false;
        cudaError_t err = cudaSuccess;
    };
    std::deque<Pending *> queue;
    bool leading = false;
    int active = 1;
    double window_s = 50e-6;
    int sms = 0, device = 0;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> pool;            // events free for reuse
    std::map<cudaEvent_t, int> waiting;       // batch event -> submitters still to wait on it
    int64_t launches = 0, jobs = 0;
    int max_jobs = 0;
};

OzBatcher *ozb_create(int device, int sms, double window_s) {
    OzBatcher *b = new (std::nothrow) OzBatcher();
    if (!b) return nullptr;
    b->device = device;
    b->sms = sms;
    b->window_s = window_s;
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return nullptr;
    }
    return b;
}

void ozb_destroy(OzBatcher *b) {
    if (!b) return;
    cudaStreamSynchronize(b->st);
    for (cudaEvent_t e : b->pool) cudaEventDestroy(e);
    for (auto &kv : b->waiting) cudaEventDestroy(kv.first);
    cudaStreamDestroy(b->st);
    delete b;
}

void ozb_set_window(OzBatcher *b, double window_s) {
    std::lock_guard<std::mutex> lk(b->mu);
    b->window_s = window_s;
}

void ozb_set_active(OzBatcher *b, int n) {
    std::lock_guard<std::mutex> lk(b->mu);
    b->active = std::max(1, n);
    b->cv.notify_all();
}

void ozb_counts(OzBatcher *b, int64_t *launches, int64_t *jobs, int *max_jobs) {
    std::lock_guard<std::mutex> lk(b->mu);
    *launches = b->launches;
    *jobs = b->jobs;
    *max_jobs = b->max_jobs;
}

namespace {

// The per-thread event a submitter records when its operands are ready.
cudaEvent_t ready_event() {
    thread_local cudaEvent_t ev = nullptr;
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ev = nullptr;
    }
    return ev;
}

// Run job (with its kernel configuration) through the batcher; returns after
// `st` waits for the launch that contains it.
cudaError_t ozb_run(OzBatcher *b, const OzJob &job, int cfg, cudaStream_t st) {
    OzBatcher::Pending me;
    me.job = job;
    me.cfg = cfg;
    me.ready = ready_event();
    if (!me.ready) return cudaErrorUnknown;
    cudaError_t e = cudaEventRecord(me.ready, st);
    if (e != cudaSuccess) return e;
    std::unique_lock<std::mutex> lk(b->mu);
    b->queue.push_back(&me);
    b->cv.notify_all();
    while (!me.launched) {
        if (b->leading) {
            b->cv.wait(lk);
            continue;
        }
        // lead: wait for company, then launch what is queued
        b->leading = true;
        const auto t_end = std::chrono::steady_clock::now() +
                           std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                               std::chrono::duration<double>(b->window_s));
        while ((int)b->queue.size() < b->active &&
               b->cv.wait_until(lk, t_end) != std::cv_status::timeout) {
        }
        std::vector<OzBatcher::Pending *> take;
        const int cfg0 = b->queue.front()->cfg;
        for (auto it = b->queue.begin(); it != b->queue.end() && (int)take.size() < kMaxJobs;) {
            if ((*it)->cfg == cfg0) {
                take.push_back(*it);
                it = b->queue.erase(it);
            } else {
                ++it;
            }
        }
        cudaEvent_t done = nullptr;
        if (!b->pool.empty()) {
            done = b->pool.back();
            b->pool.pop_back();
        }
        lk.unlock();
        OzBatch bt;
        memset(&bt, 0, sizeof bt);
        int u = 0;
        for (size_t k = 0; k < take.size(); k++) {
            bt.job[k] = take[k]->job;
            bt.job[k].unit0 = u;
            u += take[k]->job.args.tx * take[k]->job.args.ty * take[k]->job.args.tz;
        }
        bt.njobs = (int)take.size();
        bt.units = u;
        cudaError_t le = cudaSuccess;
        if (!done && cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
            le = cudaGetLastError();
            done = nullptr;
        }
        for (size_t k = 0; k < take.size() && le == cudaSuccess; k++)
            le = cudaStreamWaitEvent(b->st, take[k]->ready, 0);
        if (le == cudaSuccess) le = launch_batch(bt, cfg0, b->sms, b->st);
        if (le == cudaSuccess) le = cudaEventRecord(done, b->st);
        lk.lock();
        for (auto *p : take) {
            p->launched = true;
            p->err = le;
            p->done = (le == cudaSuccess) ? done : nullptr;
        }
        if (le == cudaSuccess) {
            b->waiting[done] = (int)take.size();
            b->launches++;
            b->jobs += (int64_t)take.size();
            b->max_jobs = std::max(b->max_jobs, (int)take.size());
        } else if (done) {
            b->pool.push_back(done);
        }
        b->leading = false;
        b->cv.notify_all();
    }
    const cudaError_t err = me.err;
    cudaEvent_t done = me.done;
    lk.unlock();
    if (err != cudaSuccess) return err;
    e = cudaStreamWaitEvent(st, done, 0);
    lk.lock();
    if (--b->waiting[done] == 0) {
        b->waiting.erase(done);
        b->pool.push_back(done);
    }
    return e;
}

}  // namespace

cudaError_t ozaki_zgemm(const OzakiH &oh, int n, const z_t *Y, int64_t ldy, z_t *C, int64_t ldc,
                        const GemmEpi &ep, void *bslices, int *F, ChaseScalars *sc, int level,
                        z_t *partials, size_t partial_bytes, int sms, cudaStream_t st,
                        cudaEvent_t ev0, cudaEvent_t ev1, OzBatcher *batcher) {
    if (n <= 0) return cudaSuccess;
    const int64_t N = oh.N, Np = oh.Np;
    const int mp = (n + kW - 1) / kW * kW;
    k_fill_int<<<(mp + 255) / 256, 256, 0, st>>>(F, mp, INT_MIN);
    bse_count_launches(1);
    // half storage: the slices of T Y (H Y = T (S (T Y)))
    const double *rs = oh.tri ? oh.t : nullptr;
    dim3 ge((unsigned)std::min<int64_t>((N + 255) / 256, 16), (unsigned)n);
    k_col_exponent<<<ge, 256, 0, st>>>(N, n, Y, ldy, F, sc, rs);
    bse_count_launches(1);
    dim3 gs((unsigned)((Np + 255) / 256), (unsigned)mp);
    k_slice_y<<<gs, 256, 0, st>>>(N, Np, n, mp, Y, ldy, F, (uint16_t *)bslices, rs);
    bse_count_launches(1);
    CUtensorMap tmB;
    if (!make_map(&tmB, bslices, (uint64_t)mp, (uint64_t)(kS * 3 * (Np / kKC)), kW))
        return cudaErrorInvalidValue;
    OzArgs a{};
    a.M = N;
    a.n = n;
    a.mp = mp;
    a.nchunks = (int)(Np / kKC);
    a.E = oh.E;
    a.F = F;
    a.sc = sc;
    const int tx = mp / kW, ty = (int)(Np / kBM);
    const int best = choose_splits(tx * ty, a.nchunks, n, N, partial_bytes, sms);
    if (best < 1) return cudaErrorInvalidValue;
    a.csplit = (a.nchunks + best - 1) / best;
    const int nsplit = (a.nchunks + a.csplit - 1) / a.csplit;
    a.P = (unsigned long long *)partials;
    a.wait_ns = oh.wait_ns;
    a.tx = tx;
    a.ty = ty;
    a.tz = nsplit;
    a.nslots = oh.tri ? (int)((Np / kBM) * (Np / kBM + 1)) : 0;
    const CUtensorMap &tmA = *(const CUtensorMap *)oh.tmap;
    OzBatch one = single(tmA, tmB, a);
    if (oh.tri) one.job[0].tmA2 = *(const CUtensorMap *)oh.tmap2;
    const int cfg = level | (oh.tri ? kOzTri : 0);
    cudaError_t e;
    if (batcher) {
        e = ozb_run(batcher, one.job[0], cfg, st);   // launched with other solvers' products
    } else {
        if (ev0) cudaEventRecord(ev0, st);
        e = launch_batch(one, cfg, sms, st);
        if (ev1) cudaEventRecord(ev1, st);
    }
    if (e != cudaSuccess) return e;
    dim3 gr((unsigned)((N + 255) / 256), (unsigned)n);
    k_split_reduce<<<gr, 256, 0, st>>>(N, n, nsplit, a.P, a.E, a.F, ep, Y, ldy, C, ldc,
                                       oh.tri ? oh.t : nullptr);
    bse_count_launches(1);
    return cudaGetLastError();
}

size_t ozaki_gen_a_bytes(int64_t M, int64_t K) {
    const int64_t Mp = (M + kBM - 1) / kBM * kBM, Kp = (K + kKC - 1) / kKC * kKC;
    return (size_t)kS * 2 * Mp * Kp * 2;
}

size_t ozaki_gen_b_bytes(int64_t K, int n) {
    const int64_t Kp = (K + kKC - 1) / kKC * kKC;
    const int64_t mp = (n + kW - 1) / kW * kW;
    return (size_t)kS * 3 * mp * Kp * 2;
}

cudaError_t ozaki_gemm(int64_t M, int n, int64_t K, const z_t *A, int64_t lda, int ah,
                       const z_t *B, int64_t ldb, int mode, const z_t *D, int64_t ldd,
                       double shift, int hermitize, z_t *C, int64_t ldc, const OzGemmWork &w,
                       ChaseScalars *sc, int sms, cudaStream_t st) {
    if (M <= 0 || n <= 0) return cudaSuccess;
    if (K <= 0 || (mode == OZ_GRAM && M != n)) return cudaErrorInvalidValue;
    const int64_t Mp = (M + kBM - 1) / kBM * kBM, Kp = (K + kKC - 1) / kKC * kKC;
    const int mp = (n + kW - 1) / kW * kW;
    if (ozaki_gen_a_bytes(M, K) > w.a_bytes || Mp > w.e_len || ozaki_gen_b_bytes(K, n) > w.b_bytes ||
        mp > w.f_len)
        return cudaErrorInvalidValue;
    // exponents and slices of op(A): rows of A, or columns of A for A^H
    k_fill_int<<<(unsigned)((Mp + 255) / 256), 256, 0, st>>>(w.E, (int)Mp, INT_MIN);
    if (ah) {
        dim3 ge((unsigned)std::min<int64_t>((K + 255) / 256, 16), (unsigned)M);
        k_col_exponent<<<ge, 256, 0, st>>>(K, (int)M, A, lda, w.E, sc);
        dim3 gs((unsigned)((Kp + 255) / 256), (unsigned)Mp);
        k_slice_ah<<<gs, 256, 0, st>>>(M, Mp, K, Kp, A, lda, w.E, (uint16_t *)w.A);
    } else {
        const int cpb = 256;
        dim3 g1((unsigned)((M + 255) / 256), (unsigned)((K + cpb - 1) / cpb));
        k_row_exponent<<<g1, 256, 0, st>>>(M, K, A, lda, w.E, cpb, sc);
        dim3 g2((unsigned)(Kp / 32), (unsigned)(Mp / 32));
        k_slice_h<<<g2, dim3(32, 8), 0, st>>>(M, Mp, K, Kp, A, lda, w.E, (uint16_t *)w.A);
    }
    // exponents and slices of B (K x n)
    k_fill_int<<<(mp + 255) / 256, 256, 0, st>>>(w.F, mp, INT_MIN);
    dim3 ge((unsigned)std::min<int64_t>((K + 255) / 256, 16), (unsigned)n);
    k_col_exponent<<<ge, 256, 0, st>>>(K, n, B, ldb, w.F, sc);
    dim3 gs((unsigned)((Kp + 255) / 256), (unsigned)mp);
    k_slice_y<<<gs, 256, 0, st>>>(K, Kp, n, mp, B, ldb, w.F, (uint16_t *)w.B);
    bse_count_launches(6);
    CUtensorMap tmA, tmB;
    if (!make_map(&tmA, w.A, (uint64_t)Mp, (uint64_t)(kS * 2 * (Kp / kKC)), kBM) ||
        !make_map(&tmB, w.B, (uint64_t)mp, (uint64_t)(kS * 3 * (Kp / kKC)), kW))
        return cudaErrorInvalidValue;
    OzArgs a{};
    a.M = M;
    a.n = n;
    a.mp = mp;
    a.nchunks = (int)(Kp / kKC);
    a.E = w.E;
    a.F = w.F;
    a.sc = sc;
    const int tx = mp / kW, ty = (int)(Mp / kBM);
    const int best = choose_splits(tx * ty, a.nchunks, n, M, w.p_bytes, sms);
    if (best < 1) return cudaErrorInvalidValue;
    a.csplit = (a.nchunks + best - 1) / best;
    const int nsplit = (a.nchunks + a.csplit - 1) / a.csplit;
    a.P = (unsigned long long *)w.P;
    a.wait_ns = w.wait_ns;
    a.tx = tx;
    a.ty = ty;
    a.tz = nsplit;
    cudaError_t e = launch_batch(single(tmA, tmB, a), OZ_S6, sms, st);
    if (e != cudaSuccess) return e;
    dim3 gr((unsigned)((M + 255) / 256), (unsigned)n);
    k_gen_reduce<<<gr, 256, 0, st>>>(M, n, nsplit, a.P, a.E, a.F, mode, D, ldd, shift, hermitize, C, ldc);
    bse_count_launches(1);
    return cudaGetLastError();
}
