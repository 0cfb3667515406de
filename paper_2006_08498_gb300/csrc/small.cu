// Single-CTA kernels for the small (m x m, m = nev + nex <= 512) dense
// problems of the ChASE iteration:
//   - Cholesky G = R^H R and the triangular inverse R^{-1} (Cholesky QR of
//     the filtered block; Supplement, "QR" item),
//   - the Hermitian eigensolver of the Rayleigh quotient G = Q^H H Q
//     (Supplement, "RR" item: the reduced problem): Householder reduction
//     to Hermitian tridiagonal form, a diagonal phase that makes it real,
//     the implicit symmetric QR iteration with Wilkinson shift (Golub & Van
//     Loan, Sec. 8.3) and back-transformation,
//   - the Lanczos spectral estimate from the small tridiagonals (Supplement,
//     "Lanczos" item), and
//   - the per-iteration update: locking, the damped interval, the
//     per-vector degrees of Eq. (S1) and their sort.
// They run on one SM and read/write global memory (L2 resident at these
// sizes).  Failures set an error word instead of trapping.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kST = 1024;                 // threads of the small kernels
constexpr int kSW = kST / 32;             // warps
constexpr int kMaxN = 512;                // largest reduced problem
static_assert(kSW == 32, "block_sum sums one partial per lane");

__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {            // one warp sums the partials; FP64 issue is scarce
        const double s = warp_sum(red[lane]);
        if (lane == 0) red[kSW] = s;
    }
    __syncthreads();
    return red[kSW];
}

// ------------------------------------------------------------ Cholesky
__global__ void __launch_bounds__(kST) k_cholesky(int n, z_t *G, int64_t ld, ChaseScalars *sc) {
    __shared__ int failed;
    __shared__ double rjj_s;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    if (threadIdx.x == 0) failed = 0;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        if (warp == 0) {
            double s = 0.0;
            for (int k = lane; k < j; k += 32) s += zabs2(G[k + (int64_t)j * ld]);
            s = warp_sum(s);
            if (lane == 0) {
                const double d = G[j + (int64_t)j * ld].x - s;
                if (!(d > 0.0)) {
                    failed = 1;
                    set_error(sc, DEV_CHOL_FAIL, j);
                } else {
                    rjj_s = sqrt(d);
                    G[j + (int64_t)j * ld] = zmk(rjj_s, 0.0);
                }
            }
        }
        __syncthreads();
        if (failed) return;
        const double inv = 1.0 / rjj_s;
        for (int i = j + 1 + warp; i < n; i += kSW) {
            z_t s = zmk(0.0, 0.0);
            for (int k = lane; k < j; k += 32)
                zcfma(s, G[k + (int64_t)j * ld], G[k + (int64_t)i * ld]);
            s.x = warp_sum(s.x);
            s.y = warp_sum(s.y);
            if (lane == 0) G[j + (int64_t)i * ld] = zscale(zsub(G[j + (int64_t)i * ld], s), inv);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += kST) {
        const int i = e % n, j = e / n;
        if (i > j) G[i + (int64_t)j * ld] = zmk(0.0, 0.0);
    }
}


// Cholesky with the upper triangle in shared memory (n <= kCholSmemN):
// packed column-major, element (i, j), i <= j, at j (j + 1) / 2 + i.  The
// same left-looking order as k_cholesky; every dot product now reads shared
// memory instead of L2, which was what bounded the global version.
constexpr int kCholSmemN = 160;

__device__ __forceinline__ int upk(int i, int j) { return j * (j + 1) / 2 + i; }

__global__ void __launch_bounds__(kST)
k_cholesky_smem(int n, z_t *G, int64_t ld, ChaseScalars *sc) {
    extern __shared__ z_t U[];
    __shared__ int failed;
    __shared__ double rjj_s;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    if (threadIdx.x == 0) failed = 0;
    for (int e = threadIdx.x; e < n * n; e += kST) {
        const int i = e % n, j = e / n;
        if (i <= j) U[upk(i, j)] = G[i + (int64_t)j * ld];
    }
    __syncthreads();
    for (int j = 0; j < n; j++) {
        const z_t *cj = U + upk(0, j);
        if (warp == 0) {
            double s = 0.0;
            for (int k = lane; k < j; k += 32) s += zabs2(cj[k]);
            s = warp_sum(s);
            if (lane == 0) {
                const double d = cj[j].x - s;
                if (!(d > 0.0)) {
                    failed = 1;
                    set_error(sc, DEV_CHOL_FAIL, j);
                } else {
                    rjj_s = sqrt(d);
                    U[upk(j, j)] = zmk(rjj_s, 0.0);
                }
            }
        }
        __syncthreads();
        if (failed) return;
        const double inv = 1.0 / rjj_s;
        for (int i = j + 1 + warp; i < n; i += kSW) {
            const z_t *ci = U + upk(0, i);
            z_t s = zmk(0.0, 0.0);
            for (int k = lane; k < j; k += 32) zcfma(s, cj[k], ci[k]);
            s.x = warp_sum(s.x);
            s.y = warp_sum(s.y);
            if (lane == 0) U[upk(j, i)] = zscale(zsub(U[upk(j, i)], s), inv);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += kST) {
        const int i = e % n, j = e / n;
        G[i + (int64_t)j * ld] = (i <= j) ? U[upk(i, j)] : zmk(0.0, 0.0);
    }
}

// X = R^{-1} for upper triangular R with a real positive diagonal: one warp
// per column j (8 per CTA, as many CTAs as needed), column-oriented back
// substitution of R x = e_j with x in shared memory and the reciprocals of
// the diagonal computed once per CTA.
__global__ void __launch_bounds__(256)
k_trinv_cols(int n, const z_t *__restrict__ R, int64_t ldr, z_t *X, int64_t ldx) {
    extern __shared__ double smt[];
    double *rinv = smt;                                   // n
    z_t *xs = (z_t *)(smt + ((n + 1) & ~1));              // 8 x n
    const int lane = threadIdx.x % 32, wl = threadIdx.x / 32;
    for (int k = threadIdx.x; k < n; k += blockDim.x) rinv[k] = 1.0 / R[k + (int64_t)k * ldr].x;
    __syncthreads();
    const int j = blockIdx.x * 8 + wl;
    if (j >= n) return;
    z_t *x = xs + (int64_t)wl * n;
    for (int r = lane; r < n; r += 32) x[r] = zmk(r == j ? 1.0 : 0.0, 0.0);
    __syncwarp();
    for (int k = j; k >= 0; k--) {
        const z_t xk = zscale(x[k], rinv[k]);
        __syncwarp();
        if (lane == 0) x[k] = xk;
        const z_t *rk = R + (int64_t)k * ldr;
        for (int r = lane; r < k; r += 32) x[r] = zsub(x[r], zmul(rk[r], xk));
        __syncwarp();
    }
    z_t *xo = X + (int64_t)j * ldx;
    for (int r = lane; r < n; r += 32) xo[r] = x[r];
}

// ------------------------------------------------- Hermitian eigensolver
// G = Q D Z Lambda Z^T D^H Q^H:
//   k_heev_reduce  (1 CTA)    Householder reduction to Hermitian tridiagonal
//                             form, Q = H_0 ... H_{n-2}, and the diagonal
//                             phases D that make it real: T' = D^H T D;
//   k_heev_tri     (n CTAs)   eigenvalue j of T' by multisection on Sturm
//                             counts (the 32 lanes of a warp count at 32
//                             points per step), then its eigenvector from a
//                             twisted factorization of T' - lambda I (one
//                             step of inverse iteration from the best unit
//                             vector; Dhillon & Parlett, 2004), on the
//                             unreduced block of T' that holds j;
//   k_heev_gram / k_heev_ns   one Newton-Schulz step Z <- Z (3I - Z^T Z)/2
//                             (n^3 work spread over SMs), which restores
//                             orthogonality lost between close eigenvalues;
//   k_heev_check              residuals |T' z - lambda z| of every column;
//   k_heev_chase / k_heev_rotate  only when a residual check failed (near
//                             multiple eigenvalues inside one unreduced
//                             block): implicit symmetric QR with Wilkinson
//                             shift (Golub & Van Loan, Sec. 8.3) on one
//                             thread, its rotations logged and replayed on
//                             the rows of Z across CTAs;
//   k_heev_back    (n/4 CTAs) ascending order and Y = Q D Z, one warp per
//                             column.
// FP64 issue is slow on this part (one SM does about 2 FP64 FMA per clock,
// shared by its warps), so the work is spread over many SMs wherever it can
// be and the serial parts keep their FP64 instruction count small.
struct HeevWork {
    z_t *V;        // n x n Householder vectors (column k from row k+1)
    double *tau;   // n
    z_t *esub;     // n   complex subdiagonal of T
    z_t *delta;    // n   phases
    z_t *p;        // n
    double *d, *e; // n, n: the real tridiagonal
    double *lam;   // n   eigenvalues (position order)
    double *Z;     // n x n real, row-major: eigenvector j in column j
    double *S1, *S2;  // n x n scratch
    int2 *sweeps;  // (p, q) of every sweep (fallback path)
    double2 *rot;  // (c, s) of every rotation, sweep after sweep
    int *nsweeps;  // 1
    int *flag;     // 1: a residual check failed, take the QR path
};

// Log capacity: sweeps <= 60 n (the per-eigenvalue sweep limit), rotations
// <= 12 n^2 (the QR iteration with Wilkinson shift takes about 2 sweeps per
// eigenvalue, i.e. about n^2 rotations; more is reported as no convergence).
__host__ __device__ inline int64_t heev_max_sweeps(int n) { return 60 * (int64_t)n; }
__host__ __device__ inline int64_t heev_max_rot(int n) { return 12 * (int64_t)n * n + 4096; }

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

__host__ __device__ inline HeevWork heev_layout(int n, void *base) {
    char *p = (char *)base;
    HeevWork w;
    const size_t nn = (size_t)n * n;
    w.V = (z_t *)p; p += align256(nn * sizeof(z_t));
    w.tau = (double *)p; p += align256(n * sizeof(double));
    w.esub = (z_t *)p; p += align256(n * sizeof(z_t));
    w.delta = (z_t *)p; p += align256(n * sizeof(z_t));
    w.p = (z_t *)p; p += align256(n * sizeof(z_t));
    w.d = (double *)p; p += align256(n * sizeof(double));
    w.e = (double *)p; p += align256(n * sizeof(double));
    w.lam = (double *)p; p += align256(n * sizeof(double));
    w.Z = (double *)p; p += align256(nn * sizeof(double));
    w.S1 = (double *)p; p += align256(nn * sizeof(double));
    w.S2 = (double *)p; p += align256(nn * sizeof(double));
    w.sweeps = (int2 *)p; p += align256(heev_max_sweeps(n) * sizeof(int2));
    w.rot = (double2 *)p; p += align256(heev_max_rot(n) * sizeof(double2));
    w.nsweeps = (int *)p; p += align256(sizeof(int));
    w.flag = (int *)p; p += align256(sizeof(int));
    return w;
}

__host__ __device__ inline size_t heev_bytes(int n) {
    const size_t nn = (size_t)n * n;
    return align256(nn * sizeof(z_t)) + align256(n * sizeof(double)) +
           3 * align256(n * sizeof(z_t)) + 3 * align256(n * sizeof(double)) +
           3 * align256(nn * sizeof(double)) + align256(heev_max_sweeps(n) * sizeof(int2)) +
           align256(heev_max_rot(n) * sizeof(double2)) + 2 * align256(sizeof(int));
}

__global__ void __launch_bounds__(kST)
k_heev_reduce(int n, z_t *A, int64_t lda, HeevWork w) {
    __shared__ double red[kSW + 1];
    __shared__ double s_tau, s_K;
    __shared__ z_t s_beta;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;

    // Householder reduction: trailing block B = A[k+1:, k+1:]
    for (int k = 0; k + 1 < n; k++) {
        const int L = n - k - 1;
        const z_t *x = A + (k + 1) + (int64_t)k * lda;
        double part = 0.0;
        for (int i = tid; i < L; i += kST) part += zabs2(x[i]);
        const double alpha = sqrt(block_sum(part, red));
        z_t *v = w.V + (k + 1) + (int64_t)k * n;
        if (L == 1 || alpha == 0.0) {
            if (tid == 0) { w.esub[k] = x[0]; w.tau[k] = 0.0; }
            __syncthreads();
            continue;
        }
        if (tid == 0) {
            const z_t x0 = x[0];
            const double ax0 = sqrt(zabs2(x0));
            const z_t ph = (ax0 > 0.0) ? zscale(x0, 1.0 / ax0) : zmk(1.0, 0.0);
            s_beta = zscale(ph, -alpha);
            // v^H v = 2 alpha (alpha + |x0|), so tau = 1 / (alpha (alpha + |x0|))
            s_tau = 1.0 / (alpha * (alpha + ax0));
            w.esub[k] = s_beta;
            w.tau[k] = s_tau;
        }
        __syncthreads();
        for (int i = tid; i < L; i += kST) v[i] = (i == 0) ? zsub(x[0], s_beta) : x[i];
        __syncthreads();
        const double t = s_tau;
        z_t *B = A + (k + 1) + (int64_t)(k + 1) * lda;
        // p_i = t sum_j B[i,j] v_j = t sum_j conj(B[j,i]) v_j (column i of B)
        for (int i = warp; i < L; i += kSW) {
            z_t s = zmk(0.0, 0.0);
            const z_t *bc = B + (int64_t)i * lda;
            for (int j = lane; j < L; j += 32) zcfma(s, bc[j], v[j]);
            s.x = warp_sum(s.x);
            s.y = warp_sum(s.y);
            if (lane == 0) w.p[i] = zscale(s, t);
        }
        __syncthreads();
        double vp = 0.0;   // Re(v^H p)
        for (int i = tid; i < L; i += kST) {
            const z_t vi = v[i], pi = w.p[i];
            vp += vi.x * pi.x + vi.y * pi.y;
        }
        vp = block_sum(vp, red);
        if (tid == 0) s_K = 0.5 * t * vp;
        __syncthreads();
        for (int i = tid; i < L; i += kST) w.p[i] = zsub(w.p[i], zscale(v[i], s_K));
        __syncthreads();
        // B -= v q^H + q v^H: computed on the lower triangle (column j by warp,
        // rows i >= j by lane) and mirrored to the upper one
        for (int j = warp; j < L; j += kSW) {
            const z_t vj = v[j], qj = w.p[j];
            for (int i = j + lane; i < L; i += 32) {
                const z_t vi = v[i], qi = w.p[i];
                z_t b = B[i + (int64_t)j * lda];
                b = zsub(b, zmul(vi, zconj(qj)));
                b = zsub(b, zmul(qi, zconj(vj)));
                if (i == j) b.y = 0.0;
                B[i + (int64_t)j * lda] = b;
                if (i != j) B[j + (int64_t)i * lda] = zconj(b);
            }
        }
        __syncthreads();
    }
    // real tridiagonal T' = D^H T D
    for (int k = tid; k < n; k += kST) {
        w.d[k] = A[k + (int64_t)k * lda].x;
        w.e[k] = (k + 1 < n) ? sqrt(zabs2(w.esub[k])) : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        w.delta[0] = zmk(1.0, 0.0);
        for (int k = 0; k + 1 < n; k++) {
            const double ae = w.e[k];
            w.delta[k + 1] = (ae > 0.0) ? zmul(w.delta[k], zscale(w.esub[k], 1.0 / ae)) : w.delta[k];
        }
    }
}

// The same reduction spread over a thread-block cluster of C CTAs (one per
// SM).  FP64 issue on one SM bounds the single-CTA version, so the trailing
// block is distributed: global column j lives in the shared memory of CTA
// j mod C, packed (rows j..n-1).  Step k of Sec. "RR" reduction:
//   the owner of column k forms v_k and tau_k and publishes them in its
//   shared memory; cluster barrier;
//   every CTA reads v_k, forms its partial of B v over the columns it
//   holds (a column axpy for rows >= j and a dot for the mirrored upper part);
//   cluster barrier;
//   every CTA sums the C partials in rank order (the same p everywhere), forms
//   q = p - (tau/2)(v^H p) v and updates its own columns; the owner of column
//   k + 1 then forms v_{k+1}.
// Control flow is uniform across the cluster (tau is read from the owner by
// every CTA), so every thread reaches every cluster barrier.
constexpr int kHhT = 256;                 // threads per CTA
constexpr int kHhW = kHhT / 32;
constexpr int kHhMaxCols = 64;            // own columns of one CTA (n <= 512, C >= 8)

__device__ double hh_block_sum(double v, double *red) {
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = (lane < kHhW) ? red[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) red[kHhW] = s;
    }
    __syncthreads();
    return red[kHhW];
}

template <int C>
__host__ __device__ constexpr int hh_cols(int n, int c) { return (c < n) ? (n - c + C - 1) / C : 0; }
// start of local column l of rank c in the packed store
template <int C>
__host__ __device__ constexpr int hh_base(int n, int c, int l) { return l * n - C * l * (l - 1) / 2 - c * l; }

template <int C>
__global__ void __launch_bounds__(kHhT)
k_heev_reduce_cl(int n, const z_t *A, int64_t lda, HeevWork w) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ z_t Bl[];                 // own columns, packed
    __shared__ z_t s_vo[2][kMaxN];              // v published by the column owner
    __shared__ z_t s_pp[kMaxN];                 // this CTA's partial of B v
    __shared__ z_t s_v[kMaxN], s_q[kMaxN];
    __shared__ z_t s_t[kHhMaxCols];
    __shared__ double s_tau[2];
    __shared__ double red[kHhW + 1];
    __shared__ z_t s_beta;
    const int c = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int ncol = hh_cols<C>(n, c);

    for (int l = 0; l < ncol; l++) {
        const int j = l * C + c;
        z_t *col = Bl + hh_base<C>(n, c, l);
        for (int r = j + tid; r < n; r += kHhT) col[r - j] = A[r + (int64_t)j * lda];
    }
    __syncthreads();

    // Householder vector of column k (called by every thread of its owner)
    auto house = [&](int k) {
        const int L = n - k - 1;
        const z_t *x = Bl + hh_base<C>(n, c, k / C) + 1;   // rows k+1 .. n-1
        double part = 0.0;
        for (int i = tid; i < L; i += kHhT) part += zabs2(x[i]);
        const double alpha = sqrt(hh_block_sum(part, red));
        if (tid == 0) {
            const z_t x0 = x[0];
            double tau = 0.0;
            z_t beta = x0;
            if (L > 1 && alpha != 0.0) {
                const double ax0 = sqrt(zabs2(x0));
                const z_t ph = (ax0 > 0.0) ? zscale(x0, 1.0 / ax0) : zmk(1.0, 0.0);
                beta = zscale(ph, -alpha);
                tau = 1.0 / (alpha * (alpha + ax0));   // 2 / (v^H v)
            }
            w.esub[k] = beta;
            w.tau[k] = tau;
            s_beta = beta;
            s_tau[k & 1] = tau;
        }
        __syncthreads();
        if (s_tau[k & 1] != 0.0) {
            z_t *vg = w.V + (k + 1) + (int64_t)k * n;
            for (int i = tid; i < L; i += kHhT) {
                const z_t vi = (i == 0) ? zsub(x[0], s_beta) : x[i];
                s_vo[k & 1][i] = vi;
                vg[i] = vi;
            }
        }
    };

    if (c == 0 && n >= 2) house(0);
    for (int k = 0; k + 1 < n; k++) {
        const int L = n - k - 1, b0 = k + 1, o = k % C;
        cl.sync();                                            // v_k published
        const double tau = *cl.map_shared_rank(&s_tau[k & 1], o);
        const int l0 = (b0 > c) ? (b0 - c + C - 1) / C : 0;  // first own column >= b0
        if (tau != 0.0) {
            const z_t *vo = cl.map_shared_rank(&s_vo[k & 1][0], o);
            for (int i = tid; i < L; i += kHhT) s_v[i] = vo[i];
            __syncthreads();
            // mirrored part: t_j = sum_{r > j} conj(B_rj) v_r for own columns j
            for (int l = l0 + warp; l < ncol; l += kHhW) {
                const int j = l * C + c;
                const z_t *col = Bl + hh_base<C>(n, c, l);
                z_t s = zmk(0.0, 0.0);
                for (int r = j + 1 + lane; r < n; r += 32) zcfma(s, col[r - j], s_v[r - b0]);
                s.x = warp_sum(s.x);
                s.y = warp_sum(s.y);
                if (lane == 0) s_t[l] = s;
            }
            // lower part: s_r = sum_{own j <= r} B_rj v_j
            for (int i = tid; i < L; i += kHhT) {
                const int r = b0 + i;
                z_t s = zmk(0.0, 0.0);
                for (int l = l0; l < ncol; l++) {
                    const int j = l * C + c;
                    if (j > r) break;
                    zfma(s, Bl[hh_base<C>(n, c, l) + (r - j)], s_v[j - b0]);
                }
                s_pp[i] = s;
            }
            __syncthreads();
            for (int i = tid; i < L; i += kHhT) {
                const int r = b0 + i;
                if (r % C == c) s_pp[i] = zadd(s_pp[i], s_t[r / C]);
            }
        }
        cl.sync();                                            // partials published
        if (tau != 0.0) {
            for (int i = tid; i < L; i += kHhT) {
                z_t s = zmk(0.0, 0.0);
                for (int cc = 0; cc < C; cc++) s = zadd(s, cl.map_shared_rank(s_pp, cc)[i]);
                s_q[i] = zscale(s, tau);                      // p = tau B v
            }
            double vp = 0.0;   // Re(v^H p)
            for (int i = tid; i < L; i += kHhT) vp += s_v[i].x * s_q[i].x + s_v[i].y * s_q[i].y;
            const double K = 0.5 * tau * hh_block_sum(vp, red);
            for (int i = tid; i < L; i += kHhT) s_q[i] = zsub(s_q[i], zscale(s_v[i], K));
            __syncthreads();
            // B -= v q^H + q v^H on the own columns (rows >= j)
            for (int l = l0 + warp; l < ncol; l += kHhW) {
                const int j = l * C + c;
                z_t *col = Bl + hh_base<C>(n, c, l);
                const z_t vj = s_v[j - b0], qj = s_q[j - b0];
                for (int r = j + lane; r < n; r += 32) {
                    const z_t vr = s_v[r - b0], qr = s_q[r - b0];
                    z_t bb = col[r - j];
                    bb.x -= vr.x * qj.x + vr.y * qj.y + qr.x * vj.x + qr.y * vj.y;
                    bb.y -= vr.y * qj.x - vr.x * qj.y + qr.y * vj.x - qr.x * vj.y;
                    if (r == j) bb.y = 0.0;
                    col[r - j] = bb;
                }
            }
            __syncthreads();
        }
        if (k + 2 < n && c == (k + 1) % C) house(k + 1);
    }
    for (int l = tid; l < ncol; l += kHhT) w.d[l * C + c] = Bl[hh_base<C>(n, c, l)].x;
    __threadfence();
    cl.sync();
    if (c == 0) {
        for (int k = tid; k < n; k += kHhT) w.e[k] = (k + 1 < n) ? sqrt(zabs2(__ldcg(&w.esub[k]))) : 0.0;
        __syncthreads();
        if (tid == 0) {
            w.delta[0] = zmk(1.0, 0.0);
            for (int k = 0; k + 1 < n; k++) {
                const double ae = w.e[k];
                w.delta[k + 1] = (ae > 0.0) ? zmul(w.delta[k], zscale(__ldcg(&w.esub[k]), 1.0 / ae)) : w.delta[k];
            }
        }
    }
}

template <int C>
size_t hh_dyn_bytes(int n) { return (size_t)hh_base<C>(n, 0, hh_cols<C>(n, 0)) * sizeof(z_t); }

// One-time set-up of a cluster kernel of C CTAs (called once per kernel
// under std::call_once, so concurrent solver threads never see a half-set
// attribute): non-portable cluster size for C > 8, the largest dynamic
// shared memory any call may use, and a check that one such cluster fits.
// Returns that byte limit, or 0 when the cluster form cannot run.
template <int C>
size_t cluster_setup(const void *kernel, size_t max_bytes, int threads) {
    if (C > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = max_bytes;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return 0;
    }
    return max_bytes;
}

template <int C, class... Args>
cudaError_t cluster_launch(void (*kernel)(Args...), size_t bytes, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kHhT);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Launches the clustered reduction with C CTAs if the cluster fits (shared
// memory, co-residency); returns cudaErrorNotSupported when it does not.
template <int C>
cudaError_t hh_launch(int n, const z_t *A, int64_t lda, const HeevWork &hw, cudaStream_t st) {
    constexpr size_t kStatic = (size_t)(5 * kMaxN + kHhMaxCols + 1) * sizeof(z_t) + 64 * sizeof(double);
    static std::once_flag once[kMaxDevices];
    static size_t limits[kMaxDevices];
    const int dev = current_device();
    if (dev < 0) return cudaErrorNotSupported;
    size_t &limit = limits[dev];
    std::call_once(once[dev], [&limit] {
        limit = cluster_setup<C>((const void *)k_heev_reduce_cl<C>,
                                 std::min(hh_dyn_bytes<C>(kMaxN), (size_t)227 * 1024 - kStatic), kHhT);
    });
    const size_t bytes = hh_dyn_bytes<C>(n);
    if (limit == 0 || bytes > limit) return cudaErrorNotSupported;
    return cluster_launch<C>(k_heev_reduce_cl<C>, bytes, st, n, A, lda, hw);
}

// Cholesky G = U^H U (Sec. "QR": the Gram matrix of the filtered block) on a
// cluster of C CTAs, right-looking: step j takes the pivot from the owner of
// column j, forms row j of U on every CTA's own columns, publishes it, and
// every CTA applies the rank-one update to the trailing upper triangle of
// its columns.  The single-CTA versions are bound by FP64 issue on one SM
// (dot products of short rows, a warp reduction each); here the work is
// element-wise and spread over C SMs.  Column j (rows 0..j) of the upper
// triangle lives in the shared memory of CTA j mod C.
template <int C>
__host__ __device__ constexpr int ch_cols(int n, int c) { return (c < n) ? (n - c + C - 1) / C : 0; }
template <int C>
__host__ __device__ constexpr int ch_base(int c, int l) { return C * l * (l - 1) / 2 + (c + 1) * l; }

template <int C>
__global__ void __launch_bounds__(kHhT)
k_cholesky_cl(int n, z_t *G, int64_t ld, ChaseScalars *sc) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ z_t Uc[];                 // own columns, rows 0..j
    __shared__ z_t s_row[kMaxN];                // row j of U on the own columns (by column)
    __shared__ z_t s_u[kMaxN];                  // row j of U, gathered
    const int c = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int ncol = ch_cols<C>(n, c);
    for (int l = 0; l < ncol; l++) {
        const int j = l * C + c;
        z_t *col = Uc + ch_base<C>(c, l);
        for (int r = tid; r <= j; r += kHhT) col[r] = G[r + (int64_t)j * ld];
    }
    cl.sync();
    for (int j = 0; j < n; j++) {
        const int o = j % C;
        // pivot: G(j, j) after j earlier updates, read from its owner; every
        // CTA takes the same decision, so all leave together on a failure
        const double d = cl.map_shared_rank(Uc, o)[ch_base<C>(o, j / C) + j].x;
        if (!(d > 0.0)) {
            if (c == 0 && tid == 0) set_error(sc, DEV_CHOL_FAIL, j);
            cl.sync();                          // nobody still reads this CTA's memory
            return;
        }
        const double rjj = sqrt(d), inv = 1.0 / rjj;
        const int l0 = (j + 1 > c) ? (j + 1 - c + C - 1) / C : 0;   // own columns > j
        for (int l = l0 + tid; l < ncol; l += kHhT) {
            z_t *col = Uc + ch_base<C>(c, l);
            const z_t u = zscale(col[j], inv);
            col[j] = u;
            s_row[l * C + c] = u;
        }
        cl.sync();                              // row j published, pivot read everywhere
        if (o == c && tid == 0) Uc[ch_base<C>(c, j / C) + j] = zmk(rjj, 0.0);
        for (int i = j + 1 + tid; i < n; i += kHhT) s_u[i] = cl.map_shared_rank(s_row, i % C)[i];
        __syncthreads();
        // G(i1, i2) -= conj(U(j, i1)) U(j, i2), j < i1 <= i2, own columns i2
        for (int l = l0 + warp; l < ncol; l += kHhW) {
            const int i2 = l * C + c;
            z_t *col = Uc + ch_base<C>(c, l);
            const z_t u2 = s_u[i2];
            for (int i1 = j + 1 + lane; i1 <= i2; i1 += 32) {
                const z_t u1 = s_u[i1];
                z_t g = col[i1];
                g.x -= u1.x * u2.x + u1.y * u2.y;
                g.y -= u1.x * u2.y - u1.y * u2.x;
                col[i1] = g;
            }
        }
        cl.sync();                              // updates done; s_row free again
    }
    for (int l = 0; l < ncol; l++) {
        const int j = l * C + c;
        const z_t *col = Uc + ch_base<C>(c, l);
        for (int r = tid; r < n; r += kHhT) G[r + (int64_t)j * ld] = (r <= j) ? col[r] : zmk(0.0, 0.0);
    }
}

template <int C>
size_t ch_dyn_bytes(int n) {
    int m = 0;
    for (int c = 0; c < C; c++) m = max(m, ch_base<C>(c, ch_cols<C>(n, c)));
    return (size_t)m * sizeof(z_t);
}

// Launches the clustered Cholesky with C CTAs if the cluster fits;
// cudaErrorNotSupported otherwise.
template <int C>
cudaError_t ch_launch(int n, z_t *G, int64_t ld, ChaseScalars *sc, cudaStream_t st) {
    constexpr size_t kStatic = (size_t)(2 * kMaxN) * sizeof(z_t) + 64;
    static std::once_flag once[kMaxDevices];
    static size_t limits[kMaxDevices];
    const int dev = current_device();
    if (dev < 0) return cudaErrorNotSupported;
    size_t &limit = limits[dev];
    std::call_once(once[dev], [&limit] {
        limit = cluster_setup<C>((const void *)k_cholesky_cl<C>,
                                 std::min(ch_dyn_bytes<C>(kMaxN), (size_t)227 * 1024 - kStatic), kHhT);
    });
    const size_t bytes = ch_dyn_bytes<C>(n);
    if (limit == 0 || bytes > limit) return cudaErrorNotSupported;
    return cluster_launch<C>(k_cholesky_cl<C>, bytes, st, n, G, ld, sc);
}

// Deflation test shared by every path: e_k is negligible next to its
// diagonal neighbours.
__device__ __forceinline__ bool tri_split(const double *d, const double *e, int k) {
    return fabs(e[k]) <= 0x1.0p-52 * (fabs(d[k]) + fabs(d[k + 1]));
}

// Number of eigenvalues below x of the unreduced block d[0..nb), e2[0..nb-1)
// (Sturm count with the pivots q_k of the LDL^T factorization of T - x I).
__device__ __forceinline__ int sturm_count(int nb, const double *d, const double *e2, double x,
                                           double pivmin) {
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    int c = q < 0.0;
    for (int k = 1; k < nb; k++) {
        q = (d[k] - x) - e2[k - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < 0.0;
    }
    return c;
}

// Eigenpair j (j = position in T', i.e. local index j - start of the
// unreduced block that holds position j).  One warp per CTA.
__global__ void __launch_bounds__(32) k_heev_tri(int n, HeevWork w) {
    __shared__ double sd[kMaxN], se[kMaxN], se2[kMaxN];
    __shared__ double s_l[kMaxN], s_dp[kMaxN], s_z[kMaxN];   // twisted factorization of lane 0
    const int j = blockIdx.x, lane = threadIdx.x;
    if (j == 0 && lane == 0) *w.flag = 0;
    for (int k = lane; k < n; k += 32) {
        sd[k] = w.d[k];
        se[k] = (k + 1 < n) ? w.e[k] : 0.0;
    }
    __syncwarp();
    // the unreduced block [bs, be) holding j
    int bs = 0, be = n;
    for (int k = lane; k + 1 < n; k += 32) {
        if (tri_split(sd, se, k)) {
            if (k < j) bs = max(bs, k + 1);
            else be = min(be, k + 1);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        bs = max(bs, __shfl_xor_sync(0xffffffffu, bs, o));
        be = min(be, __shfl_xor_sync(0xffffffffu, be, o));
    }
    const int nb = be - bs, li = j - bs;
    const double *d = sd + bs;
    double emax = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double ek = (k >= bs && k + 1 < be) ? se[k] : 0.0;
        se2[k] = ek * ek;
        emax = fmax(emax, fabs(ek));
    }
    for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    __syncwarp();
    const double *e2 = se2 + bs;
    const double pivmin = 0x1.0p-1000 * fmax(1.0, emax * emax);
    // Gershgorin interval of the block
    double lo = INFINITY, hi = -INFINITY;
    for (int k = lane; k < nb; k += 32) {
        const double r = (k > 0 ? sqrt(e2[k - 1]) : 0.0) + (k + 1 < nb ? sqrt(e2[k]) : 0.0);
        lo = fmin(lo, d[k] - r);
        hi = fmax(hi, d[k] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double widen = 0x1.0p-50 * fmax(fabs(lo), fabs(hi)) + 2.0 * pivmin;
    double a = lo - widen, b = hi + widen;
    // multisection: 32 points per step, the interval shrinks 33-fold
    for (int it = 0; it < 24; it++) {
        if (b - a <= 0x1.0p-52 * fmax(fabs(a), fabs(b)) + 2.0 * pivmin) break;
        const double h = (b - a) / 33.0;
        const double x = a + (lane + 1) * h;
        const int c = sturm_count(nb, d, e2, x, pivmin);
        const unsigned above = __ballot_sync(0xffffffffu, c > li);
        if (above == 0u) {
            a = a + 32.0 * h;
        } else {
            const int l = __ffs(above) - 1;
            const double bn = a + (l + 1) * h;
            a = (l > 0) ? a + l * h : a;
            b = bn;
        }
    }
    const double lam = 0.5 * (a + b);
    if (lane != 0) return;
    w.lam[j] = lam;
    // twisted factorization of T' - lam I on the block: L+ D+ L+^T from the
    // top (multipliers l, pivots dp), U- D- U-^T from the bottom, twist index
    // r = argmin |gamma_k|; all in shared memory (this loop is serial, and
    // global loads behind its own stores would each pay L2 latency)
    double piv = d[0] - lam;
    for (int k = 0; k < nb; k++) {
        if (fabs(piv) < pivmin) piv = -pivmin;
        s_dp[k] = piv;
        if (k + 1 < nb) {
            const double ek = se[bs + k];
            const double l = ek / piv;
            s_l[k] = l;
            piv = (d[k + 1] - lam) - l * ek;
        }
    }
    double dm = d[nb - 1] - lam;
    if (fabs(dm) < pivmin) dm = -pivmin;
    int r = nb - 1;
    double gmin = fabs(s_dp[nb - 1]);   // gamma_{nb-1} = dp_{nb-1}
    // u_k (k >= 1) kept in s_z[k] until the vector pass overwrites it
    for (int k = nb - 2; k >= 0; k--) {
        const double ek = se[bs + k];
        const double u = ek / dm;
        s_z[k + 1] = u;
        dm = (d[k] - lam) - u * ek;
        if (fabs(dm) < pivmin) dm = -pivmin;
        const double g = fabs(s_dp[k] + dm - (d[k] - lam));
        if (g < gmin) { gmin = g; r = k; }
    }
    // z_r = 1; z_k = -l_k z_{k+1} above r, z_k = -u_k z_{k-1} below r
    double nrm = 1.0, zk = 1.0;
    for (int k = r - 1; k >= 0; k--) {
        zk = -s_l[k] * zk;
        s_z[k] = zk;
        nrm = fma(zk, zk, nrm);
    }
    s_z[r] = 1.0;
    zk = 1.0;
    for (int k = r + 1; k < nb; k++) {
        zk = -s_z[k] * zk;
        s_z[k] = zk;
        nrm = fma(zk, zk, nrm);
    }
    const double inv = 1.0 / sqrt(nrm);
    double *z = w.Z;
    const int64_t ld = n;
    for (int k = 0; k < n; k++) {
        const int64_t ix = (int64_t)k * ld + j;
        z[ix] = (k >= bs && k < be) ? s_z[k - bs] * inv : 0.0;
    }
}

// M = Z^T Z (S1 = M; 16 x 16 tiles of M per 256-thread CTA)
__global__ void __launch_bounds__(256) k_heev_gram(int n, HeevWork w) {
    const int r = blockIdx.y * 16 + threadIdx.y, c = blockIdx.x * 16 + threadIdx.x;
    if (*w.flag) return;
    if (r >= n || c >= n) return;
    double s = 0.0;
    for (int k = 0; k < n; k++) s = fma(w.Z[(int64_t)k * n + r], w.Z[(int64_t)k * n + c], s);
    w.S1[(int64_t)r * n + c] = s;
}

// S2 = Z (3 I - M) / 2, one Newton-Schulz step towards the orthogonal polar
// factor of Z
__global__ void __launch_bounds__(256) k_heev_ns(int n, HeevWork w) {
    const int r = blockIdx.y * 16 + threadIdx.y, c = blockIdx.x * 16 + threadIdx.x;
    if (*w.flag) return;
    if (r >= n || c >= n) return;
    double s = 0.0;
    for (int k = 0; k < n; k++) s = fma(w.Z[(int64_t)r * n + k], w.S1[(int64_t)k * n + c], s);
    w.S2[(int64_t)r * n + c] = 1.5 * w.Z[(int64_t)r * n + c] - 0.5 * s;
}

// Every column of S2 must pass |T' z - lam z|_inf <= tol |T'| and
// | |z|^2 - 1 | <= tol; any failure (or a NaN) raises the flag for the QR
// path.  After one Newton-Schulz step the orthogonality error E satisfies
// |E_ij| <= sqrt(E_ii E_jj) to leading order, so the column norms bound it
// (identical vectors, from eigenvalues equal to working precision inside
// one block, come out as zero columns and fail here).  One warp per column.
__global__ void __launch_bounds__(128) k_heev_check(int n, HeevWork w, double tol) {
    const int lane = threadIdx.x % 32, c = blockIdx.x * 4 + threadIdx.x / 32;
    if (c >= n) return;
    const double lam = w.lam[c];
    double tn = 0.0, res = 0.0, nrm = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double em = k > 0 ? w.e[k - 1] : 0.0, ek = k + 1 < n ? w.e[k] : 0.0;
        tn = fmax(tn, fabs(w.d[k]) + fabs(em) + fabs(ek));
        const double zk = w.S2[(int64_t)k * n + c];
        double t = (w.d[k] - lam) * zk;
        if (k > 0) t += em * w.S2[(int64_t)(k - 1) * n + c];
        if (k + 1 < n) t += ek * w.S2[(int64_t)(k + 1) * n + c];
        res = fmax(res, fabs(t));
        if (!(t == t)) res = INFINITY;
        nrm = fma(zk, zk, nrm);
    }
    nrm = warp_sum(nrm);
    for (int o = 16; o > 0; o >>= 1) {
        tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
        res = fmax(res, __shfl_xor_sync(0xffffffffu, res, o));
    }
    if (lane == 0 && !(res <= tol * tn && fabs(nrm - 1.0) <= tol)) atomicExch(w.flag, 1);
}

// Z <- S2 once every column passed
__global__ void __launch_bounds__(256) k_heev_accept(int n, HeevWork w) {
    if (*w.flag) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int64_t)n * n) w.Z[i] = w.S2[i];
}

// Implicit QR on the real tridiagonal (one thread).  d and e live in shared
// memory; the d[k], e[k] of the current chase step are carried in registers.
// A rotation is taken from rsqrt(x^2 + z^2): entries here are bounded by
// the norm of the reduced matrix, so the squares neither overflow nor lose
// anything that matters to the deflation test.
__global__ void k_heev_chase(int n, HeevWork w, ChaseScalars *sc) {
    __shared__ double d[kMaxN], e[kMaxN];
    if (threadIdx.x != 0 || !*w.flag) return;
    for (int k = 0; k < n; k++) { d[k] = w.d[k]; e[k] = w.e[k]; }
    const double eps = 0x1.0p-52;
    const int64_t max_sw = heev_max_sweeps(n), max_rot = heev_max_rot(n);
    int64_t nsw = 0, nrot = 0;
    int q = n - 1, sweeps = 0;
    bool failed = false;
    while (q > 0) {
        if (fabs(e[q - 1]) <= eps * (fabs(d[q - 1]) + fabs(d[q]))) {
            e[q - 1] = 0.0;
            q--;
            sweeps = 0;
            continue;
        }
        int p = q - 1;
        while (p > 0 && fabs(e[p - 1]) > eps * (fabs(d[p - 1]) + fabs(d[p]))) p--;
        if (p > 0) e[p - 1] = 0.0;
        if (++sweeps > 60 || nsw >= max_sw || nrot + (q - p) > max_rot) {
            failed = true;
            break;
        }
        const double hd = (d[q - 1] - d[q]) / 2.0, bq = e[q - 1];
        const double den = hd + copysign(hypot(hd, bq), hd);
        const double mu = (den != 0.0) ? d[q] - bq * bq / den : d[q] - fabs(bq);
        w.sweeps[nsw++] = make_int2(p, q);
        double2 *rl = w.rot + nrot;
        nrot += q - p;
        double x = d[p] - mu, z = e[p];
        double ak = d[p], bk = e[p];
        for (int k = p; k < q; k++) {
            const double ak1 = d[k + 1];
            const double en = (k < q - 1) ? e[k + 1] : 0.0;
            const double t2 = fma(x, x, z * z);
            double c = 1.0, sn = 0.0, r = 0.0;
            if (t2 > 0x1.0p-1000) {
                const double ir = rsqrt(t2);
                c = x * ir;
                sn = -z * ir;
                r = t2 * ir;
            } else if (t2 > 0.0) {       // tiny: the scaled form
                r = hypot(x, z);
                c = x / r;
                sn = -z / r;
            }
            if (k > p) e[k - 1] = r;
            const double cc = c * c, ss = sn * sn, cs = c * sn;
            const double csb = 2.0 * cs * bk;
            d[k] = fma(cc, ak, fma(ss, ak1, -csb));
            const double dk1 = fma(ss, ak, fma(cc, ak1, csb));
            const double ek = fma(cs, ak - ak1, (cc - ss) * bk);
            e[k] = ek;
            if (k < q - 1) {
                x = ek;
                z = -sn * en;
                bk = c * en;
            }
            ak = dk1;
            rl[k - p] = make_double2(c, sn);
        }
        d[q] = ak;
    }
    for (int k = 0; k < n; k++) w.lam[k] = d[k];
    *w.nsweeps = failed ? -1 : (int)nsw;
    if (failed) set_error(sc, DEV_EIG_NOCONV, n);
}

// Z = I, then every logged rotation applied to the rows of Z: lane = row.
// The CTA's 32 rows sit in shared memory as Zs[k][lane].
__global__ void __launch_bounds__(32) k_heev_rotate(int n, HeevWork w) {
    extern __shared__ double Zs[];
    const int lane = threadIdx.x, row = blockIdx.x * 32 + lane;
    if (!*w.flag) return;
    const int nsw = *w.nsweeps;
    if (nsw < 0) return;
    for (int k = 0; k < n; k++) Zs[k * 32 + lane] = (k == row) ? 1.0 : 0.0;
    __syncwarp();
    const double2 *rot = w.rot;
    for (int s = 0; s < nsw; s++) {
        const int2 pq = w.sweeps[s];
        const int p = pq.x, q = pq.y;
        double carry = Zs[p * 32 + lane];
#pragma unroll 4
        for (int k = p; k < q; k++) {
            const double2 r = rot[k - p];
            const double zk1 = Zs[(k + 1) * 32 + lane];
            Zs[k * 32 + lane] = r.x * carry - r.y * zk1;
            carry = fma(r.y, carry, r.x * zk1);
        }
        Zs[q * 32 + lane] = carry;
        rot += q - p;
    }
    __syncwarp();
    if (row < n)
        for (int k = 0; k < n; k++) w.Z[(int64_t)row * n + k] = Zs[k * 32 + lane];
}

// Eigenvalues ascending (stable rank) and column rank[c] of Y = Q D Z[:, c];
// one warp per column c, its vector in shared memory.
__global__ void __launch_bounds__(128)
k_heev_back(int n, HeevWork w, double *wout, z_t *Y, int64_t ldy) {
    __shared__ z_t ys[4][kMaxN];
    const int lane = threadIdx.x % 32, wl = threadIdx.x / 32;
    const int c = blockIdx.x * 4 + wl;
    if (c >= n || (*w.flag && *w.nsweeps < 0)) return;
    const double dc = w.lam[c];
    int r = 0;
    for (int j = lane; j < n; j += 32) {
        const double dj = w.lam[j];
        r += (dj < dc) || (dj == dc && j < c);
    }
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    z_t *y = ys[wl];
    for (int i = lane; i < n; i += 32) y[i] = zscale(w.delta[i], w.Z[(int64_t)i * n + c]);
    __syncwarp();
    for (int k = n - 2; k >= 0; k--) {
        const double t = w.tau[k];
        if (t == 0.0) continue;
        const z_t *v = w.V + (k + 1) + (int64_t)k * n;
        const int L = n - k - 1;
        z_t s = zmk(0.0, 0.0);
        for (int i = lane; i < L; i += 32) zcfma(s, v[i], y[k + 1 + i]);
        s.x = warp_sum(s.x);
        s.y = warp_sum(s.y);
        s = zscale(s, t);
        for (int i = lane; i < L; i += 32) y[k + 1 + i] = zsub(y[k + 1 + i], zmul(s, v[i]));
        __syncwarp();
    }
    z_t *yo = Y + (int64_t)r * ldy;
    for (int i = lane; i < n; i += 32) yo[i] = y[i];
    if (lane == 0) wout[r] = dc;
}

// ------------------------------------------------- Lanczos estimate
constexpr int kMaxK = 64;
constexpr int kMaxRuns = 8;

// Implicit QR of one small tridiagonal, accumulating only the first row of
// the eigenvector matrix (enough for the weights tau_i = z_{0,i}^2).
__device__ int tridiag_first_row(int n, double *d, double *e, double *z0) {
    const double eps = 0x1.0p-52;
    for (int i = 0; i < n; i++) z0[i] = (i == 0) ? 1.0 : 0.0;
    int q = n - 1, sweeps = 0;
    while (q > 0) {
        if (fabs(e[q - 1]) <= eps * (fabs(d[q - 1]) + fabs(d[q]))) {
            e[q - 1] = 0.0;
            q--;
            sweeps = 0;
            continue;
        }
        int p = q - 1;
        while (p > 0 && fabs(e[p - 1]) > eps * (fabs(d[p - 1]) + fabs(d[p]))) p--;
        if (p > 0) e[p - 1] = 0.0;
        if (++sweeps > 60) return -1;
        const double hd = (d[q - 1] - d[q]) / 2.0, bq = e[q - 1];
        const double den = hd + copysign(hypot(hd, bq), hd);
        const double mu = (den != 0.0) ? d[q] - bq * bq / den : d[q] - fabs(bq);
        double x = d[p] - mu, z = e[p];
        for (int k = p; k < q; k++) {
            const double r = hypot(x, z);
            const double c = (r == 0.0) ? 1.0 : x / r;
            const double s = (r == 0.0) ? 0.0 : -z / r;
            if (k > p) e[k - 1] = r;
            const double ak = d[k], ak1 = d[k + 1], bk = e[k];
            d[k] = c * c * ak - 2.0 * c * s * bk + s * s * ak1;
            d[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * ak1;
            e[k] = c * s * (ak - ak1) + (c * c - s * s) * bk;
            if (k < q - 1) {
                x = e[k];
                z = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            const double zk = z0[k], zk1 = z0[k + 1];
            z0[k] = c * zk - s * zk1;
            z0[k + 1] = s * zk + c * zk1;
        }
    }
    return 0;
}

__global__ void k_lanczos_finalize(int k, int nl, int64_t N, int m, const double *alpha,
                                   const double *beta, ChaseScalars *sc) {
    __shared__ double th[kMaxRuns * kMaxK], tw[kMaxRuns * kMaxK], up[kMaxRuns];
    const int l = threadIdx.x;
    if (l < nl) {
        double d[kMaxK], e[kMaxK], z0[kMaxK];
        for (int i = 0; i < k; i++) d[i] = alpha[i * nl + l];
        for (int i = 0; i + 1 < k; i++) e[i] = beta[i * nl + l];
        if (tridiag_first_row(k, d, e, z0) != 0) set_error(sc, DEV_EIG_NOCONV, l);
        double dmax = d[0];
        for (int i = 0; i < k; i++) {
            th[l * k + i] = d[i];
            tw[l * k + i] = z0[i] * z0[i];
            dmax = fmax(dmax, d[i]);
        }
        up[l] = dmax + fabs(beta[(k - 1) * nl + l]);
    }
    __syncthreads();
    if (l != 0) return;
    const int P = k * nl;
    double b = up[0], mu1 = th[0];
    for (int r = 1; r < nl; r++) b = fmax(b, up[r]);
    for (int i = 0; i < P; i++) mu1 = fmin(mu1, th[i]);
    // pooled Ritz values in ascending order (insertion sort, stable)
    for (int i = 1; i < P; i++) {
        const double x = th[i], wt = tw[i];
        int j = i - 1;
        while (j >= 0 && th[j] > x) { th[j + 1] = th[j]; tw[j + 1] = tw[j]; j--; }
        th[j + 1] = x;
        tw[j + 1] = wt;
    }
    const double scale = (double)N / (double)nl;
    double cnt = 0.0, prev_cnt = 0.0, mum = th[P - 1];
    for (int i = 0; i < P; i++) {
        prev_cnt = cnt;
        cnt += tw[i] * scale;
        if (cnt >= (double)m) {
            mum = (i == 0) ? th[0]
                           : th[i - 1] + ((double)m - prev_cnt) * (th[i] - th[i - 1]) / (cnt - prev_cnt);
            break;
        }
    }
    sc->beta = b;
    sc->mu_1 = mu1;
    sc->mu_m = mum;
    sc->norm_est = fmax(fabs(mu1), fabs(b));
    sc->alpha = mum;
    sc->lower = mu1;
}

// ------------------------------------------------- per-iteration update
__device__ int degree_of(double theta, double r, double c, double e, double tol, int deg_max) {
    const double t = (theta - c) / e;
    const double at = fabs(t);
    int d;
    if (at <= 1.0) {
        d = deg_max;
    } else {
        const double rho = at + sqrt(t * t - 1.0);
        if (r <= tol) {
            d = 2;
        } else {
            const double q = ceil(log(r / tol) / log(rho));
            d = (q <= (double)deg_max) ? (int)q : deg_max;   // NaN -> deg_max
            if (d < 2) d = 2;
        }
    }
    d += d & 1;
    return d < deg_max ? d : deg_max;
}

__global__ void k_chase_update(int m_act, int nev, double tol, int deg_max,
                               const double *theta, const double *resid, int *deg, int *perm,
                               ChaseScalars *sc) {
    __shared__ int nl_s;
    __shared__ double c_s, e_s;
    __shared__ int dtmp[kMaxN];
    if (threadIdx.x == 0) {
        int nl = 0;
        const int locked = sc->locked;
        while (nl < m_act && locked + nl < nev && resid[nl] <= tol) nl++;
        nl_s = nl;
        sc->new_locked = nl;
        sc->locked = locked + nl;
        sc->alpha = theta[m_act - 1];
        sc->lower = fmin(sc->lower, theta[0]);
        c_s = (sc->alpha + sc->beta) / 2.0;
        e_s = (sc->beta - sc->alpha) / 2.0;
        sc->m_act = m_act - nl;
    }
    __syncthreads();
    const int nl = nl_s, mu = m_act - nl;
    for (int j = threadIdx.x; j < mu; j += blockDim.x)
        dtmp[j] = degree_of(theta[nl + j], resid[nl + j], c_s, e_s, tol, deg_max);
    __syncthreads();
    for (int j = threadIdx.x; j < mu; j += blockDim.x) {
        const int dj = dtmp[j];
        int r = 0;
        for (int i = 0; i < mu; i++) r += (dtmp[i] < dj) || (dtmp[i] == dj && i < j);
        deg[r] = dj;
        perm[nl + r] = nl + j;
    }
    for (int j = threadIdx.x; j < nl; j += blockDim.x) perm[j] = j;
}

}  // namespace

cudaError_t launch_cholesky(int n, z_t *G, int64_t ld, ChaseScalars *sc, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n <= kMaxN) {
        cudaError_t ce = ch_launch<16>(n, G, ld, sc, st);
        if (ce == cudaErrorNotSupported) ce = ch_launch<8>(n, G, ld, sc, st);
        if (ce != cudaErrorNotSupported) {
            bse_count_launches(1);
            return ce;
        }
    }
    if (n <= kCholSmemN) {
        const int bytes = (kCholSmemN * (kCholSmemN + 1) / 2) * (int)sizeof(z_t);
        static std::once_flag once[kMaxDevices];
        static cudaError_t attr[kMaxDevices];
        const cudaError_t ae = smem_attr_once(once, attr, (const void *)k_cholesky_smem, bytes);
        if (ae != cudaSuccess) return ae;
        k_cholesky_smem<<<1, kST, (size_t)(n * (n + 1) / 2) * sizeof(z_t), st>>>(n, G, ld, sc);
    } else {
        k_cholesky<<<1, kST, 0, st>>>(n, G, ld, sc);
    }
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trinv(int n, const z_t *R, int64_t ldr, z_t *X, int64_t ldx, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t bytes = (size_t)((n + 1) & ~1) * sizeof(double) + (size_t)8 * n * sizeof(z_t);
    static std::once_flag once[kMaxDevices];
    static cudaError_t attr[kMaxDevices];
    const int maxb = (int)(((kMaxN + 1) & ~1) * sizeof(double) + 8 * kMaxN * sizeof(z_t));
    {
        const cudaError_t ae = smem_attr_once(once, attr, (const void *)k_trinv_cols, maxb);
        if (ae != cudaSuccess) return ae;
    }
    k_trinv_cols<<<(n + 7) / 8, 256, bytes, st>>>(n, R, ldr, X, ldx);
    bse_count_launches(1);
    return cudaGetLastError();
}

size_t heev_work_bytes(int n) { return heev_bytes(n); }

cudaError_t launch_heev(int n, z_t *A, int64_t lda, double *w, z_t *Y, int64_t ldy, void *work,
                        ChaseScalars *sc, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > kMaxN) return cudaErrorInvalidValue;
    const HeevWork hw = heev_layout(n, work);
    cudaError_t he = hh_launch<16>(n, A, lda, hw, st);
    if (he == cudaErrorNotSupported) he = hh_launch<8>(n, A, lda, hw, st);
    if (he == cudaErrorNotSupported) {
        k_heev_reduce<<<1, kST, 0, st>>>(n, A, lda, hw);
        he = cudaGetLastError();
    }
    if (he != cudaSuccess) return he;
    k_heev_tri<<<n, 32, 0, st>>>(n, hw);
    const dim3 tg((n + 15) / 16, (n + 15) / 16), tb(16, 16);
    k_heev_gram<<<tg, tb, 0, st>>>(n, hw);
    k_heev_ns<<<tg, tb, 0, st>>>(n, hw);
    k_heev_check<<<(n + 3) / 4, 128, 0, st>>>(n, hw, 64.0 * 0x1.0p-52 * n);
    k_heev_accept<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, st>>>(n, hw);
    k_heev_chase<<<1, 32, 0, st>>>(n, hw, sc);
    const size_t zs = (size_t)32 * n * sizeof(double);
    static std::once_flag once[kMaxDevices];
    static cudaError_t attr[kMaxDevices];
    {
        const cudaError_t ae = smem_attr_once(once, attr, (const void *)k_heev_rotate, 32 * kMaxN * (int)sizeof(double));
        if (ae != cudaSuccess) return ae;
    }
    k_heev_rotate<<<(n + 31) / 32, 32, zs, st>>>(n, hw);
    k_heev_back<<<(n + 3) / 4, 128, 0, st>>>(n, hw, w, Y, ldy);
    bse_count_launches(9);
    return cudaGetLastError();
}

cudaError_t launch_lanczos_finalize(int k, int nl, int64_t N, int m, const double *alpha,
                                    const double *beta, ChaseScalars *sc, cudaStream_t st) {
    if (k < 1 || k > kMaxK || nl < 1 || nl > kMaxRuns) return cudaErrorInvalidValue;
    k_lanczos_finalize<<<1, 32, 0, st>>>(k, nl, N, m, alpha, beta, sc);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_chase_update(int m_act, int nev, double tol, int deg_max,
                                const double *theta, const double *resid, int *deg, int *perm,
                                ChaseScalars *sc, cudaStream_t st) {
    if (m_act < 1 || m_act > kMaxN) return cudaErrorInvalidValue;
    k_chase_update<<<1, 256, 0, st>>>(m_act, nev, tol, deg_max, theta, resid, deg, perm, sc);
    bse_count_launches(1);
    return cudaGetLastError();
}
