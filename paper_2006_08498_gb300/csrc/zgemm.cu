// FP64 complex dense products of the ChASE iteration.
//
// zgemm_nn: C = epi(A B).  It is the Chebyshev filter's product H Y_t with
// the three-term recurrence fused into the epilogue (Sec. 3: the filter is
// a three-term recurrence of HEMM calls; Supplement "Filter" item), the
// Rayleigh-Ritz product W = H Q and back-transforms Q Y, W Y (Supplement
// "RR" item), the triangular solve V R^{-1} of Cholesky QR and the
// locked-vector projection V -= V_L X (Supplement "QR" item).
//
// zgemm_cn: G = A^H B for tall-skinny A, B (Gram matrices of Cholesky QR,
// the projection X = V_L^H V and the Rayleigh quotient Q^H W), split over K
// with a fixed partition and a fixed-order reduction: deterministic.
//
// Arithmetic: complex products in four real FMAs (4M form), FP64
// throughout.  On GB300 FP64 issue, not memory, bounds both kernels: the
// filter product has 8 N^2 w flops over 16 N^2 + 32 N w bytes.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBK = 16;

// Thread (tr, tc) of a TRxTC grid owns rows tr + TR*a (a < TM) and
// columns tc + TC*b (b < TN) of a (TR*TM) x (TC*TN) tile.
template <int TR, int TM, int TC, int TN>
__global__ void __launch_bounds__(kThreads)
zgemm_nn_kernel(int64_t M, int64_t n, int64_t K, const z_t *__restrict__ A, int64_t lda,
                const z_t *__restrict__ B, int64_t ldb, z_t *C, int64_t ldc, GemmEpi ep) {
    static_assert(TR * TC == kThreads, "thread grid");
    constexpr int BM = TR * TM, BN = TC * TN;
    __shared__ z_t As[kBK][BM];
    __shared__ z_t Bs[kBK][BN];
    const int tid = threadIdx.x;
    const int tr = tid % TR, tc = tid / TR;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;

    z_t acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; a++)
#pragma unroll
        for (int b = 0; b < TN; b++) acc[a][b] = zmk(0.0, 0.0);

    // an upper triangular B has no rows below this tile's last column
    const int64_t Ke = (ep.b_upper && j0 + BN < K) ? j0 + BN : K;
    for (int64_t k0 = 0; k0 < Ke; k0 += kBK) {
        // A tile: BM rows x kBK columns, rows contiguous in memory
        for (int e = tid; e < BM * kBK; e += kThreads) {
            const int r = e % BM, kk = e / BM;
            const int64_t gi = i0 + r, gk = k0 + kk;
            As[kk][r] = (gi < M && gk < K) ? A[gi + gk * lda] : zmk(0.0, 0.0);
        }
        // B tile: kBK rows x BN columns
        for (int e = tid; e < BN * kBK; e += kThreads) {
            const int kk = e % kBK, c = e / kBK;
            const int64_t gk = k0 + kk, gj = j0 + c;
            Bs[kk][c] = (gk < K && gj < n) ? B[gk + gj * ldb] : zmk(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kBK; kk++) {
            z_t av[TM], bv[TN];
#pragma unroll
            for (int a = 0; a < TM; a++) av[a] = As[kk][tr + TR * a];
#pragma unroll
            for (int b = 0; b < TN; b++) bv[b] = Bs[kk][tc + TC * b];
#pragma unroll
            for (int a = 0; a < TM; a++)
#pragma unroll
                for (int b = 0; b < TN; b++) zfma(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int a = 0; a < TM; a++) {
        const int64_t gi = i0 + tr + TR * a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < TN; b++) {
            const int64_t gj = j0 + tc + TC * b;
            if (gj >= n) continue;
            z_t v = acc[a][b];
            if (ep.mode == GEMM_CHEB) {
                const z_t y = B[gi + gj * ldb];  // requires M == K: row gi of the operand
                v = zscale(zsub(v, zscale(y, ep.c)), ep.s1);
                if (ep.Yp) v = zsub(v, zscale(ep.Yp[gi + gj * ep.ldyp], ep.s2));
            } else if (ep.mode == GEMM_SUB) {
                v = zsub(ep.D[gi + gj * ep.ldd], v);
            }
            C[gi + gj * ldc] = v;
        }
    }
}

template <int TR, int TM, int TC, int TN>
cudaError_t run_nn(int64_t M, int64_t n, int64_t K, const z_t *A, int64_t lda, const z_t *B,
                   int64_t ldb, z_t *C, int64_t ldc, const GemmEpi &ep, cudaStream_t st) {
    constexpr int BM = TR * TM, BN = TC * TN;
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((n + BN - 1) / BN));
    zgemm_nn_kernel<TR, TM, TC, TN><<<grid, kThreads, 0, st>>>(M, n, K, A, lda, B, ldb, C, ldc, ep);
    bse_count_launches(1);
    return cudaGetLastError();
}

// ---- G = A^H B, split-K
constexpr int kGT = 32;    // output tile 32 x 32
constexpr int kGBK = 32;   // K step

__global__ void __launch_bounds__(kThreads)
zgemm_cn_partial(int64_t m1, int64_t m2, int64_t K, int64_t kchunk, const z_t *__restrict__ A,
                 int64_t lda, const z_t *__restrict__ B, int64_t ldb, z_t *__restrict__ P,
                 int upper) {
    __shared__ z_t As[kGBK][kGT + 1];
    __shared__ z_t Bs[kGBK][kGT + 1];
    // Hermitian product (A = B): tiles below the diagonal are mirrored
    if (upper && blockIdx.y < blockIdx.x) return;
    const int tid = threadIdx.x;
    const int ti = tid % 16, tj = tid / 16;
    const int64_t i0 = (int64_t)blockIdx.x * kGT, j0 = (int64_t)blockIdx.y * kGT;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = (kb + kchunk < K) ? kb + kchunk : K;
    z_t acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) acc[a][b] = zmk(0.0, 0.0);
    for (int64_t k0 = kb; k0 < ke; k0 += kGBK) {
        for (int e = tid; e < kGT * kGBK; e += kThreads) {
            const int kk = e % kGBK, c = e / kGBK;
            const int64_t gk = k0 + kk;
            As[kk][c] = (gk < ke && i0 + c < m1) ? A[gk + (i0 + c) * lda] : zmk(0.0, 0.0);
            Bs[kk][c] = (gk < ke && j0 + c < m2) ? B[gk + (j0 + c) * ldb] : zmk(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kGBK; kk++) {
            const z_t a0 = As[kk][ti], a1 = As[kk][ti + 16];
            const z_t b0 = Bs[kk][tj], b1 = Bs[kk][tj + 16];
            zcfma(acc[0][0], a0, b0);
            zcfma(acc[0][1], a0, b1);
            zcfma(acc[1][0], a1, b0);
            zcfma(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
    z_t *Pz = P + (int64_t)blockIdx.z * m1 * m2;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int64_t gi = i0 + ti + 16 * a, gj = j0 + tj + 16 * b;
            if (gi < m1 && gj < m2) Pz[gi + gj * m1] = acc[a][b];
        }
}

// G = sum_z P[z] in increasing z, + shift on the diagonal; optionally
// replaced by its Hermitian part (G + G^H)/2 (square G only).  upper: only
// the tiles on and above the diagonal were computed (A = B); the lower
// triangle is the conjugate of the upper one.
__global__ void zgemm_cn_reduce(int64_t m1, int64_t m2, int nsplit, const z_t *__restrict__ P,
                                z_t *G, int64_t ldg, double shift, int hermitize, int upper) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m1 * m2) return;
    const int64_t i = e % m1, j = e / m1;
    z_t s = zmk(0.0, 0.0), t = zmk(0.0, 0.0);
    if (upper) {
        const int64_t r = i <= j ? i : j, c = i <= j ? j : i;
        for (int z = 0; z < nsplit; z++) s = zadd(s, P[(int64_t)z * m1 * m2 + r + c * m1]);
        if (i > j) s.y = -s.y;
        if (i == j) s.y = 0.0;
        if (i == j) s.x += shift;
        G[i + j * ldg] = s;
        return;
    }
    for (int z = 0; z < nsplit; z++) s = zadd(s, P[(int64_t)z * m1 * m2 + i + j * m1]);
    if (hermitize) {
        for (int z = 0; z < nsplit; z++) t = zadd(t, P[(int64_t)z * m1 * m2 + j + i * m1]);
        s = zmk(0.5 * (s.x + t.x), 0.5 * (s.y - t.y));
        if (i == j) s.y = 0.0;
    }
    if (i == j) s.x += shift;
    G[i + j * ldg] = s;
}

int cn_nsplit(int64_t m1, int64_t m2, int64_t K, bool upper = false) {
    const int64_t t1 = (m1 + kGT - 1) / kGT, t2 = (m2 + kGT - 1) / kGT;
    const int64_t tiles = upper ? t1 * (t1 + 1) / 2 : t1 * t2;
    int64_t ns = (4 * 152 + tiles - 1) / tiles;           // ~4 CTAs per SM
    const int64_t maxs = (K + 255) / 256;                   // >= 256 rows per split
    if (ns > maxs) ns = maxs;
    if (ns < 1) ns = 1;
    if (ns > 512) ns = 512;
    return (int)ns;
}

}  // namespace

cudaError_t launch_zgemm_nn(int64_t M, int64_t n, int64_t K, const z_t *A, int64_t lda,
                            const z_t *B, int64_t ldb, z_t *C, int64_t ldc, const GemmEpi &ep,
                            cudaStream_t st) {
    if (M <= 0 || n <= 0) return cudaSuccess;
    if (n <= 4) return run_nn<64, 2, 4, 1>(M, n, K, A, lda, B, ldb, C, ldc, ep, st);
    if (n <= 8) return run_nn<64, 2, 4, 2>(M, n, K, A, lda, B, ldb, C, ldc, ep, st);
    if (n <= 16) return run_nn<16, 4, 16, 1>(M, n, K, A, lda, B, ldb, C, ldc, ep, st);
    if (n <= 32) return run_nn<16, 4, 16, 2>(M, n, K, A, lda, B, ldb, C, ldc, ep, st);
    // width per column tile: the smallest of 48 / 64 that wastes least
    const int64_t t64 = (n + 63) / 64, t48 = (n + 47) / 48;
    if (t48 * 48 < t64 * 64) return run_nn<16, 4, 16, 3>(M, n, K, A, lda, B, ldb, C, ldc, ep, st);
    return run_nn<16, 4, 16, 4>(M, n, K, A, lda, B, ldb, C, ldc, ep, st);
}

int64_t zgemm_cn_work_elems(int64_t m1, int64_t m2, int64_t K) {
    return (int64_t)cn_nsplit(m1, m2, K) * m1 * m2;
}

cudaError_t launch_zgemm_cn(int64_t m1, int64_t m2, int64_t K, const z_t *A, int64_t lda,
                            const z_t *B, int64_t ldb, z_t *G, int64_t ldg, double shift,
                            int hermitize, z_t *work, int64_t work_elems, cudaStream_t st) {
    if (m1 <= 0 || m2 <= 0) return cudaSuccess;
    // A^H A is Hermitian: compute the upper tiles only
    const int upper = (A == B && lda == ldb && m1 == m2) ? 1 : 0;
    int ns = cn_nsplit(m1, m2, K, upper != 0);
    if ((int64_t)ns * m1 * m2 > work_elems) ns = (int)(work_elems / (m1 * m2));
    if (ns < 1) return cudaErrorInvalidValue;
    const int64_t kchunk = (((K + ns - 1) / ns) + kGBK - 1) / kGBK * kGBK;
    dim3 grid((unsigned)((m1 + kGT - 1) / kGT), (unsigned)((m2 + kGT - 1) / kGT), (unsigned)ns);
    zgemm_cn_partial<<<grid, kThreads, 0, st>>>(m1, m2, K, kchunk, A, lda, B, ldb, work, upper);
    bse_count_launches(1);
    const int64_t tot = m1 * m2;
    zgemm_cn_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m1, m2, ns, work, G, ldg, shift,
                                                                  hermitize, upper);
    bse_count_launches(1);
    return cudaGetLastError();
}
