/*
 * Plain CPU FP64 oracle for the ChASE hot path (arXiv 2006.08498).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path: every formula here
 * is written out from its definition, slowly and in the order the
 * definition states it, so that it can be checked by eye.
 *
 * Contents
 *   - SplitMix64 as a counter-based generator (Steele, Lea, Flood, OOPSLA
 *     2014: state += 0x9E3779B97F4A7C15, then the 64-bit finaliser).
 *   - The seeded synthetic BSE Hamiltonian of Eq. (1) (Sec. 2): transition
 *     energies E_c(k) - E_v(k) on the diagonal, a rank-R repulsive exchange
 *     term (the 2*vbar term) and a screened attractive direct term (the W
 *     term) coupling only equal band pairs and decaying with |k - k'|.
 *   - Dense Hermitian eigensolver: Householder reduction to Hermitian
 *     tridiagonal form, a diagonal unitary phase that makes it real, and the
 *     implicit symmetric QR iteration with Wilkinson shift (Golub & Van Loan,
 *     Matrix Computations, Sec. 8.3) with eigenvector accumulation.
 *   - Cholesky factorisation G = R^H R of a small Hermitian matrix, used by
 *     the CholQR step of the QR phase (Supplement, "QR" item of the ChASE
 *     timing breakdown).
 *
 * Layout: every matrix is column-major, element (i, j) at a[i + j*ld];
 * complex numbers are interleaved (re, im) pairs, i.e. C99 double complex.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

/* ------------------------------------------------------------------ RNG */

/* One SplitMix64 output for a counter: the generator's state is set to
 * `key`, advanced by the golden gamma, and the finaliser is applied. */
uint64_t or_splitmix64(uint64_t key)
{
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1): the top 53 bits of the output times 2^-53.
 * The key mixes the user seed, a stream id in the top byte and an index. */
double or_uniform(uint64_t seed, uint64_t stream, uint64_t idx)
{
    uint64_t key = seed ^ (stream << 56) ^ idx;
    return (double)(or_splitmix64(key) >> 11) * 0x1.0p-53;
}

/* Seeded complex block with entries (2u-1) + i(2u'-1): column j, row i
 * uses indices 2*(j*n + i) and 2*(j*n + i) + 1 of `stream`. */
void or_random_block(uint64_t seed, uint64_t stream, int64_t n, int64_t m,
                     zc *V, int64_t ld)
{
    for (int64_t j = 0; j < m; j++)
        for (int64_t i = 0; i < n; i++) {
            uint64_t idx = 2 * (uint64_t)(j * n + i);
            double re = 2.0 * or_uniform(seed, stream, idx) - 1.0;
            double im = 2.0 * or_uniform(seed, stream, idx + 1) - 1.0;
            V[i + j * ld] = re + I * im;
        }
}

/* ------------------------------------------------- synthetic Eq. (1) H */

/* Model parameters of the synthetic Hamiltonian (energies in eV). */
typedef struct {
    double band_gap; /* E_c(k=0,c=0) - E_v(k=0,v=0) before jitter          */
    double w0;       /* strength of the screened direct term W            */
    double x0;       /* strength of the exchange term (its eigenvalue sum) */
    double jitter;   /* amplitude of the random conduction-band jitter     */
    double dispersion; /* scale of the cosine band dispersion (1 = default) */
    int rank_x;      /* rank of the exchange term                          */
} or_model;

/* Per-pair tables: transition energy dE[I], exchange vectors a[r + R*I]
 * and direct-term phases theta[I], for the pair index
 * I(k, v, c) = (k*Nv + v)*Nc + c. */
void or_bse_tables(uint64_t seed, int Nk, int Nv, int Nc, const or_model *md,
                   double *dE, zc *a, double *theta)
{
    const int64_t N = (int64_t)Nk * Nv * Nc;
    const int R = md->rank_x;
    const double two_pi = 6.283185307179586476925286766559;
    const double amp = sqrt(3.0 * md->x0 / (double)N) / sqrt(2.0);
    for (int k = 0; k < Nk; k++) {
        double s = (1.0 - cos(two_pi * (double)k / (double)Nk)) / 2.0;
        for (int v = 0; v < Nv; v++)
            for (int c = 0; c < Nc; c++) {
                int64_t Ip = ((int64_t)k * Nv + v) * Nc + c;
                double xi = 2.0 * or_uniform(seed, 1, (uint64_t)k * Nc + c) - 1.0;
                double Ec = md->band_gap / 2.0 + c + 3.0 * md->dispersion * s + md->jitter * xi;
                double Ev = -md->band_gap / 2.0 - 0.5 * v - 2.0 * md->dispersion * s;
                dE[Ip] = Ec - Ev;
                for (int r = 0; r < R; r++) {
                    uint64_t idx = 2 * ((uint64_t)R * Ip + r);
                    double u1 = 2.0 * or_uniform(seed, 2, idx) - 1.0;
                    double u2 = 2.0 * or_uniform(seed, 2, idx + 1) - 1.0;
                    a[r + (int64_t)R * Ip] = amp * u1 + I * (amp * u2);
                }
                theta[Ip] = two_pi * or_uniform(seed, 3, (uint64_t)Ip);
            }
    }
}

/* One element H_IJ with I >= J (lower triangle, including the diagonal). */
static zc bse_lower_element(int64_t Ip, int64_t Jp, int Nk, int Nv, int Nc,
                            const or_model *md, const double *dE, const zc *a,
                            const double *theta)
{
    const int R = md->rank_x;
    /* exchange: 2 * sum_r a_r(I) conj(a_r(J)) */
    zc x = 0.0;
    for (int r = 0; r < R; r++)
        x += a[r + (int64_t)R * Ip] * conj(a[r + (int64_t)R * Jp]);
    x = 2.0 * x;
    /* direct: w0 K(d(k,k')) delta_vv' delta_cc' e^{i(theta_I - theta_J)} */
    int64_t kI = Ip / ((int64_t)Nv * Nc), kJ = Jp / ((int64_t)Nv * Nc);
    int64_t bI = Ip % ((int64_t)Nv * Nc), bJ = Jp % ((int64_t)Nv * Nc);
    zc w = 0.0;
    if (bI == bJ) {
        int64_t dk = kI > kJ ? kI - kJ : kJ - kI;
        if (Nk - dk < dk) dk = Nk - dk;
        double K = 1.0 / ((double)dk * (double)dk + 0.5);
        double ph = theta[Ip] - theta[Jp];
        w = md->w0 * K * (cos(ph) + I * sin(ph));
    }
    (void)Nk;
    if (Ip == Jp) /* the diagonal is real by construction */
        return (dE[Ip] + creal(x) - creal(w)) + 0.0 * I;
    return x - w;
}

/* Full Hermitian H (N x N, column-major, leading dimension ld): the lower
 * triangle is computed, the upper triangle is its conjugate mirror. */
void or_bse_build(uint64_t seed, int Nk, int Nv, int Nc, const or_model *md,
                  zc *H, int64_t ld)
{
    const int64_t N = (int64_t)Nk * Nv * Nc;
    double *dE = malloc(sizeof(double) * N);
    double *theta = malloc(sizeof(double) * N);
    zc *a = malloc(sizeof(zc) * N * md->rank_x);
    or_bse_tables(seed, Nk, Nv, Nc, md, dE, a, theta);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < N; j++)
        for (int64_t i = j; i < N; i++) {
            zc h = bse_lower_element(i, j, Nk, Nv, Nc, md, dE, a, theta);
            H[i + j * ld] = h;
            H[j + i * ld] = conj(h);
        }
    free(dE);
    free(theta);
    free(a);
}

/* Transition energies only (the spectrum when x0 = w0 = 0). */
void or_bse_diagonal(uint64_t seed, int Nk, int Nv, int Nc, const or_model *md,
                     double *dE)
{
    const int64_t N = (int64_t)Nk * Nv * Nc;
    double *theta = malloc(sizeof(double) * N);
    zc *a = malloc(sizeof(zc) * N * (md->rank_x > 0 ? md->rank_x : 1));
    or_bse_tables(seed, Nk, Nv, Nc, md, dE, a, theta);
    free(theta);
    free(a);
}

/* ------------------------------------- real symmetric tridiagonal eig */

/* Eigenvalues (and, if Z != NULL, eigenvectors) of the real symmetric
 * tridiagonal matrix with diagonal d[0..n-1] and off-diagonal e[0..n-2]
 * (T[i+1,i] = T[i,i+1] = e[i]), by the implicit symmetric QR iteration with
 * Wilkinson shift and deflation.  Z is n x n ROW-major (Z[row*n + col]) and
 * must hold the matrix the rotations are accumulated into (the identity
 * for eigenvectors of T).  On return d holds the eigenvalues in ascending
 * order and column j of Z the matching eigenvector.  Returns 0, or -1 if an
 * eigenvalue did not converge in 60 sweeps. */
int or_tridiag_eig(int n, double *d, double *e, double *Z)
{
    const double eps = 0x1.0p-52;
    double *cs = malloc(sizeof(double) * 2 * (n > 1 ? n : 1));
    int q = n - 1, sweeps = 0, rc = 0;
    while (q > 0) {
        /* deflate converged eigenvalues at the bottom */
        if (fabs(e[q - 1]) <= eps * (fabs(d[q - 1]) + fabs(d[q]))) {
            e[q - 1] = 0.0;
            q--;
            sweeps = 0;
            continue;
        }
        /* find the top p of the unreduced block [p..q] */
        int p = q - 1;
        while (p > 0 && fabs(e[p - 1]) > eps * (fabs(d[p - 1]) + fabs(d[p])))
            p--;
        if (p > 0) e[p - 1] = 0.0;
        if (++sweeps > 60) { rc = -1; break; }
        /* Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[q] */
        double hd = (d[q - 1] - d[q]) / 2.0, bq = e[q - 1];
        double den = hd + copysign(hypot(hd, bq), hd);
        double mu = (den != 0.0) ? d[q] - bq * bq / den : d[q] - fabs(bq);
        /* implicit QR step: chase the bulge from p down to q */
        double x = d[p] - mu, z = e[p];
        for (int k = p; k < q; k++) {
            double r = hypot(x, z);
            double c = (r == 0.0) ? 1.0 : x / r;
            double s = (r == 0.0) ? 0.0 : -z / r;
            if (k > p) e[k - 1] = r;
            double ak = d[k], ak1 = d[k + 1], bk = e[k];
            d[k] = c * c * ak - 2.0 * c * s * bk + s * s * ak1;
            d[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * ak1;
            e[k] = c * s * (ak - ak1) + (c * c - s * s) * bk;
            if (k < q - 1) {
                x = e[k];
                z = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            cs[2 * (k - p)] = c;
            cs[2 * (k - p) + 1] = s;
        }
        if (Z) {
            /* Z <- Z G_p G_{p+1} ... G_{q-1}; each row independently */
#pragma omp parallel for schedule(static) if (n >= 256)
            for (int row = 0; row < n; row++) {
                double *zr = Z + (int64_t)row * n;
                for (int k = p; k < q; k++) {
                    double c = cs[2 * (k - p)], s = cs[2 * (k - p) + 1];
                    double zk = zr[k], zk1 = zr[k + 1];
                    zr[k] = c * zk - s * zk1;
                    zr[k + 1] = s * zk + c * zk1;
                }
            }
        }
    }
    free(cs);
    /* ascending order (selection sort keeps it plain) */
    for (int i = 0; i < n - 1; i++) {
        int kmin = i;
        for (int j = i + 1; j < n; j++)
            if (d[j] < d[kmin]) kmin = j;
        if (kmin != i) {
            double t = d[i]; d[i] = d[kmin]; d[kmin] = t;
            if (Z)
                for (int row = 0; row < n; row++) {
                    double *zr = Z + (int64_t)row * n;
                    double u = zr[i]; zr[i] = zr[kmin]; zr[kmin] = u;
                }
        }
    }
    return rc;
}

/* ----------------------------------------- dense Hermitian eigensolver */

/* All eigenvalues w[0..n-1] (ascending) of the Hermitian matrix A
 * (n x n, column-major, both triangles present; destroyed), and the
 * eigenvectors of the nz smallest in Zout (n x nz, column-major, ldz).
 * Steps: (1) Householder: for column k, x = A[k+1:, k], v = x - beta e1
 * with beta = -phase(x0)|x|, tau = 2/(v^H v), H_k = I - tau v v^H, and the
 * trailing block becomes H_k A H_k; (2) D = diag(delta) with
 * delta_{k+1} = delta_k * phase(T[k+1,k]) makes T real: T = D T' D^H;
 * (3) implicit QR on T'; (4) vectors Q D z with Q = H_0 H_1 ... H_{n-3}.
 * Returns 0, or -1 if the tridiagonal iteration failed. */
int or_heev(int n, zc *A, int64_t lda, double *w, zc *Zout, int64_t ldz, int nz)
{
    zc *V = calloc((size_t)n * n, sizeof(zc)); /* reflector k in column k */
    double *tau = calloc(n, sizeof(double));
    zc *esub = calloc(n, sizeof(zc));
    double *dg = malloc(sizeof(double) * n);
    zc *p = malloc(sizeof(zc) * n);
    for (int k = 0; k + 1 < n; k++) {
        int L = n - k - 1;
        zc *x = A + (k + 1) + (int64_t)k * lda;
        double alpha = 0.0;
        for (int i = 0; i < L; i++) alpha += creal(x[i] * conj(x[i]));
        alpha = sqrt(alpha);
        zc *v = V + (k + 1) + (int64_t)k * n;
        if (L == 1 || alpha == 0.0) { /* nothing to annihilate */
            esub[k] = x[0];
            tau[k] = 0.0;
            continue;
        }
        zc phase = (cabs(x[0]) > 0.0) ? x[0] / cabs(x[0]) : 1.0;
        zc beta = -phase * alpha;
        for (int i = 0; i < L; i++) v[i] = x[i];
        v[0] = x[0] - beta;
        double vv = 0.0;
        for (int i = 0; i < L; i++) vv += creal(v[i] * conj(v[i]));
        double t = 2.0 / vv;
        tau[k] = t;
        esub[k] = beta;
        /* trailing block B = A[k+1:, k+1:]: p = t B v, K = (t/2) v^H p,
         * q = p - K v, B <- B - v q^H - q v^H */
        zc *B = A + (k + 1) + (int64_t)(k + 1) * lda;
#pragma omp parallel for schedule(static) if (L >= 256)
        for (int i = 0; i < L; i++) {
            zc s = 0.0;
            for (int j = 0; j < L; j++) s += B[i + (int64_t)j * lda] * v[j];
            p[i] = t * s;
        }
        zc vp = 0.0;
        for (int i = 0; i < L; i++) vp += conj(v[i]) * p[i];
        double K = t / 2.0 * creal(vp);
        for (int i = 0; i < L; i++) p[i] = p[i] - K * v[i];
#pragma omp parallel for schedule(static) if (L >= 256)
        for (int j = 0; j < L; j++)
            for (int i = 0; i < L; i++)
                B[i + (int64_t)j * lda] -= v[i] * conj(p[j]) + p[i] * conj(v[j]);
        /* column k below the subdiagonal is now zero (kept implicit) */
    }
    for (int k = 0; k < n; k++) dg[k] = creal(A[k + (int64_t)k * lda]);
    /* phases making the tridiagonal real */
    zc *delta = malloc(sizeof(zc) * n);
    double *eoff = malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
    delta[0] = 1.0;
    for (int k = 0; k + 1 < n; k++) {
        double ae = cabs(esub[k]);
        eoff[k] = ae;
        delta[k + 1] = (ae > 0.0) ? delta[k] * (esub[k] / ae) : delta[k];
    }
    double *Z = NULL;
    if (nz > 0) {
        Z = calloc((size_t)n * n, sizeof(double));
        for (int i = 0; i < n; i++) Z[(int64_t)i * n + i] = 1.0;
    }
    int rc = or_tridiag_eig(n, dg, eoff, Z);
    for (int i = 0; i < n; i++) w[i] = dg[i];
    if (nz > 0) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = 0; j < nz; j++) {
            zc *y = Zout + (int64_t)j * ldz;
            for (int i = 0; i < n; i++) y[i] = delta[i] * Z[(int64_t)i * n + j];
            for (int k = n - 2; k >= 0; k--) {
                if (tau[k] == 0.0) continue;
                const zc *v = V + (k + 1) + (int64_t)k * n;
                int L = n - k - 1;
                zc s = 0.0;
                for (int i = 0; i < L; i++) s += conj(v[i]) * y[k + 1 + i];
                s *= tau[k];
                for (int i = 0; i < L; i++) y[k + 1 + i] -= s * v[i];
            }
        }
        free(Z);
    }
    free(V); free(tau); free(esub); free(dg); free(p); free(delta); free(eoff);
    return rc;
}

/* ------------------------------------------------------------ Cholesky */

/* G = R^H R for Hermitian positive definite G (n x n, column-major, upper
 * triangle read).  R (upper triangular, real positive diagonal) overwrites
 * the upper triangle of G; the strict lower triangle is set to zero.
 * Returns 0, or j+1 if the pivot of column j is not positive. */
int or_cholesky(int n, zc *G, int64_t ld)
{
    for (int j = 0; j < n; j++) {
        double djj = creal(G[j + (int64_t)j * ld]);
        for (int k = 0; k < j; k++) {
            zc rkj = G[k + (int64_t)j * ld];
            djj -= creal(rkj * conj(rkj));
        }
        if (!(djj > 0.0)) return j + 1;
        double rjj = sqrt(djj);
        G[j + (int64_t)j * ld] = rjj;
        for (int i = j + 1; i < n; i++) {
            zc s = G[j + (int64_t)i * ld];
            for (int k = 0; k < j; k++)
                s -= conj(G[k + (int64_t)j * ld]) * G[k + (int64_t)i * ld];
            G[j + (int64_t)i * ld] = s / rjj;
        }
    }
    for (int j = 0; j < n; j++)
        for (int i = j + 1; i < n; i++) G[i + (int64_t)j * ld] = 0.0;
    return 0;
}

/* Selected elements H[I[t], J[t]] (t < n) of the synthetic Hamiltonian,
 * without forming H (for spot checks at sizes where H is large). */
void or_bse_elements(uint64_t seed, int Nk, int Nv, int Nc, const or_model *md,
                     int64_t n, const int64_t *Iv, const int64_t *Jv, zc *out)
{
    const int64_t N = (int64_t)Nk * Nv * Nc;
    double *dE = malloc(sizeof(double) * N);
    double *theta = malloc(sizeof(double) * N);
    zc *a = malloc(sizeof(zc) * N * (md->rank_x > 0 ? md->rank_x : 1));
    or_bse_tables(seed, Nk, Nv, Nc, md, dE, a, theta);
    for (int64_t t = 0; t < n; t++) {
        int64_t i = Iv[t], j = Jv[t];
        out[t] = (i >= j) ? bse_lower_element(i, j, Nk, Nv, Nc, md, dE, a, theta)
                          : conj(bse_lower_element(j, i, Nk, Nv, Nc, md, dE, a, theta));
    }
    free(dE);
    free(theta);
    free(a);
}
