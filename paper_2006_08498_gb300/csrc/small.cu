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
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kST = 1024;                 // threads of the small kernels
constexpr int kSW = kST / 32;             // warps
constexpr int kMaxN = 512;                // largest reduced problem

__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kSW; w++) s += red[w];  // same order in every thread
    return s;
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

// ------------------------------------------------- triangular inverse
// Column j of X = R^{-1} by column-oriented back substitution of R x = e_j.
__global__ void __launch_bounds__(kST)
k_trinv(int n, const z_t *__restrict__ R, int64_t ldr, z_t *X, int64_t ldx) {
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    for (int j = warp; j < n; j += kSW) {
        z_t *x = X + (int64_t)j * ldx;
        for (int r = lane; r < n; r += 32) x[r] = zmk(r == j ? 1.0 : 0.0, 0.0);
        __syncwarp();
        for (int k = j; k >= 0; k--) {
            z_t xk;
            if (lane == 0) {
                const z_t rkk = R[k + (int64_t)k * ldr];
                const double inv = 1.0 / rkk.x;   // real positive diagonal
                xk = zscale(x[k], inv);
                x[k] = xk;
            }
            __syncwarp();
            xk = x[k];
            for (int r = lane; r < k; r += 32) {
                const z_t rk = R[r + (int64_t)k * ldr];
                x[r] = zsub(x[r], zmul(rk, xk));
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------- Hermitian eigensolver
// G = Q D Z Lambda Z^T D^H Q^H in four launches:
//   k_heev_reduce  (1 CTA)   Householder reduction to Hermitian tridiagonal
//                            form, Q = H_0 ... H_{n-2}, and the diagonal
//                            phases D that make it real: T' = D^H T D;
//   k_heev_chase   (1 thread) implicit symmetric QR with Wilkinson shift and
//                            deflation (Golub & Van Loan, Sec. 8.3) on T',
//                            eigenvalues only; the Givens rotations of every
//                            sweep are written to a log;
//   k_heev_rotate  (n/32 CTAs) replays the log on the rows of Z = I;
//   k_heev_back    (n/4 CTAs) ascending order and Y = Q D Z, one warp per
//                            column.
// FP64 issue is slow on this part (one SM does about 1.6 FP64 FMA per
// clock, and a dependent FP64 operation takes tens of clocks), so the serial
// chase keeps its dependent chain short and leaves all O(n^2)-per-sweep
// work to the rotation replay, and the O(n^3) parts run on many SMs where
// they can.
struct HeevWork {
    z_t *V;        // n x n Householder vectors (column k from row k+1)
    double *tau;   // n
    z_t *esub;     // n   complex subdiagonal of T
    z_t *delta;    // n   phases
    z_t *p;        // n
    double *d, *e; // n, n: the real tridiagonal; d holds the eigenvalues after the chase
    double *Z;     // n x n real, row-major
    int2 *sweeps;  // (p, q) of every sweep
    double2 *rot;  // (c, s) of every rotation, sweep after sweep
    int *nsweeps;  // 1
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
    w.Z = (double *)p; p += align256(nn * sizeof(double));
    w.sweeps = (int2 *)p; p += align256(heev_max_sweeps(n) * sizeof(int2));
    w.rot = (double2 *)p; p += align256(heev_max_rot(n) * sizeof(double2));
    w.nsweeps = (int *)p; p += align256(sizeof(int));
    return w;
}

__global__ void __launch_bounds__(kST)
k_heev_reduce(int n, z_t *A, int64_t lda, HeevWork w) {
    __shared__ double red[kSW];
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

// Implicit QR on the real tridiagonal (one thread).  d and e live in shared
// memory; the d[k], e[k] of the current chase step are carried in registers.
// A rotation is taken from rsqrt(x^2 + z^2): entries here are bounded by
// the norm of the reduced matrix, so the squares neither overflow nor lose
// anything that matters to the deflation test.
__global__ void k_heev_chase(int n, HeevWork w, ChaseScalars *sc) {
    __shared__ double d[kMaxN], e[kMaxN];
    if (threadIdx.x != 0) return;
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
    for (int k = 0; k < n; k++) w.d[k] = d[k];
    *w.nsweeps = failed ? -1 : (int)nsw;
    if (failed) set_error(sc, DEV_EIG_NOCONV, n);
}

// Z = I, then every logged rotation applied to the rows of Z: lane = row.
// The CTA's 32 rows sit in shared memory as Zs[k][lane].
__global__ void __launch_bounds__(32) k_heev_rotate(int n, HeevWork w) {
    extern __shared__ double Zs[];
    const int lane = threadIdx.x, row = blockIdx.x * 32 + lane;
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
    if (c >= n || *w.nsweeps < 0) return;
    const double dc = w.d[c];
    int r = 0;
    for (int j = lane; j < n; j += 32) {
        const double dj = w.d[j];
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
    k_cholesky<<<1, kST, 0, st>>>(n, G, ld, sc);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trinv(int n, const z_t *R, int64_t ldr, z_t *X, int64_t ldx, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_trinv<<<1, kST, 0, st>>>(n, R, ldr, X, ldx);
    bse_count_launches(1);
    return cudaGetLastError();
}

size_t heev_work_bytes(int n) {
    const size_t nn = (size_t)n * n;
    return align256(nn * sizeof(z_t)) + align256(n * sizeof(double)) +
           3 * align256(n * sizeof(z_t)) + 2 * align256(n * sizeof(double)) +
           align256(nn * sizeof(double)) + align256(heev_max_sweeps(n) * sizeof(int2)) +
           align256(heev_max_rot(n) * sizeof(double2)) + align256(sizeof(int));
}

cudaError_t launch_heev(int n, z_t *A, int64_t lda, double *w, z_t *Y, int64_t ldy, void *work,
                        ChaseScalars *sc, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > kMaxN) return cudaErrorInvalidValue;
    const HeevWork hw = heev_layout(n, work);
    k_heev_reduce<<<1, kST, 0, st>>>(n, A, lda, hw);
    k_heev_chase<<<1, 32, 0, st>>>(n, hw, sc);
    const size_t zs = (size_t)32 * n * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_heev_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             32 * kMaxN * (int)sizeof(double));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_heev_rotate<<<(n + 31) / 32, 32, zs, st>>>(n, hw);
    k_heev_back<<<(n + 3) / 4, 128, 0, st>>>(n, hw, w, Y, ldy);
    bse_count_launches(4);
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
