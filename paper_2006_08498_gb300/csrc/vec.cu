// Bandwidth-bound column kernels of the ChASE iteration: column norms and
// scaling (QR pre-scaling), eigenpair residuals (Supplement, "Resid" item),
// column gathers and permutations (locking and the degree sort), seeded
// start vectors, and the vector part of the Lanczos steps (Supplement,
// "Lanczos" item).
//
// Reductions over the N rows are deterministic: a fixed number of blocks,
// each owning a fixed row range, writes one partial per column; partials
// are summed in block order.  One warp reduces one column of a block's
// row range with coalesced loads and a shuffle tree.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kVT = 256;
constexpr int kWarps = kVT / 32;

// partial[b * nc + j] = sum over rows of block b of f(i, j)
template <class F>
__device__ void col_partials(int64_t N, int nc, double *partial, F f) {
    const int64_t chunk = (N + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = (r0 + chunk < N) ? r0 + chunk : N;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int j = warp; j < nc; j += kWarps) {
        double s = 0.0;
        for (int64_t i = r0 + lane; i < r1; i += 32) s += f(i, j);
        s = warp_sum(s);
        if (lane == 0) partial[(int64_t)blockIdx.x * nc + j] = s;
    }
}

__device__ __forceinline__ double sum_partials(const double *partial, int nb, int nc, int j) {
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += partial[(int64_t)b * nc + j];
    return s;
}

__global__ void __launch_bounds__(kVT)
k_col_sq(int64_t N, int nc, const z_t *__restrict__ X, int64_t ldx, double *partial) {
    col_partials(N, nc, partial, [&](int64_t i, int j) { return zabs2(X[i + j * ldx]); });
}

__global__ void k_finish_norms(int nb, int nc, const double *partial, double *out, int take_sqrt,
                               ChaseScalars *sc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nc) return;
    double s = sum_partials(partial, nb, nc, j);
    if (!isfinite(s)) set_error(sc, DEV_NONFINITE, j);
    out[j] = take_sqrt ? sqrt(s) : s;
}

__global__ void k_col_inv_scale(int64_t N, int nc, z_t *X, int64_t ldx, const double *s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= N || j >= nc) return;
    const double inv = 1.0 / s[j];
    X[i + j * ldx] = zscale(X[i + j * ldx], inv);
}

__global__ void __launch_bounds__(kVT)
k_resid(int64_t N, int nc, const z_t *__restrict__ HV, int64_t ldhv, const z_t *__restrict__ V,
        int64_t ldv, const double *__restrict__ theta, double *partial) {
    col_partials(N, nc, partial, [&](int64_t i, int j) {
        const z_t r = zsub(HV[i + j * ldhv], zscale(V[i + j * ldv], theta[j]));
        return zabs2(r);
    });
}

__global__ void k_finish_resid(int nb, int nc, const double *partial, double *r,
                               ChaseScalars *sc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nc) return;
    const double s = sum_partials(partial, nb, nc, j);
    if (!isfinite(s)) set_error(sc, DEV_NONFINITE, j);
    r[j] = sqrt(s) / sc->norm_est;
}

__global__ void k_copy_cols(int64_t N, int nc, const z_t *__restrict__ in, int64_t ldin,
                            z_t *__restrict__ out, int64_t ldout, const int *perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= N || j >= nc) return;
    const int src = perm ? perm[j] : j;
    out[i + j * ldout] = in[i + (int64_t)src * ldin];
}

__global__ void k_select_cols(int64_t N, int nc, const z_t *__restrict__ A,
                              const z_t *__restrict__ B, int64_t ld, const int *deg, int parity,
                              z_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= N || j >= nc) return;
    const z_t *src = ((deg[j] & 1) == parity) ? B : A;
    out[i + j * ld] = src[i + j * ld];
}

__global__ void k_random_block(uint64_t seed, uint64_t stream, int64_t n, int col0, z_t *V,
                               int64_t ldv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = col0 + blockIdx.y;
    if (i >= n) return;
    const uint64_t idx = 2 * (uint64_t)((int64_t)j * n + i);
    const double re = 2.0 * unif(seed, stream, idx) - 1.0;
    const double im = 2.0 * unif(seed, stream, idx + 1) - 1.0;
    V[i + (int64_t)j * ldv] = zmk(re, im);
}

// Lanczos, per column l: dot partials of Re(v^H w)
__global__ void __launch_bounds__(kVT)
k_lz_dot(int64_t N, int nl, const z_t *__restrict__ V, const z_t *__restrict__ W, int64_t ld,
         double *partial) {
    col_partials(N, nl, partial, [&](int64_t i, int j) {
        const z_t v = V[i + j * ld], w = W[i + j * ld];
        return v.x * w.x + v.y * w.y;
    });
}

// w -= a v + b vprev (a from the dot partials, b = previous beta), and
// partials of ||w||^2
__global__ void __launch_bounds__(kVT)
k_lz_update(int64_t N, int nl, const z_t *__restrict__ V, const z_t *__restrict__ Vprev,
            z_t *__restrict__ W, int64_t ld, const double *dot_partial, int nb,
            const double *__restrict__ beta_prev, double *norm_partial) {
    __shared__ double a_s[8], b_s[8];
    if (threadIdx.x < nl) {
        a_s[threadIdx.x] = sum_partials(dot_partial, nb, nl, threadIdx.x);
        b_s[threadIdx.x] = beta_prev[threadIdx.x];
    }
    __syncthreads();
    col_partials(N, nl, norm_partial, [&](int64_t i, int j) {
        const z_t v = V[i + j * ld], vp = Vprev[i + j * ld];
        z_t w = W[i + j * ld];
        w.x -= a_s[j] * v.x + b_s[j] * vp.x;
        w.y -= a_s[j] * v.y + b_s[j] * vp.y;
        W[i + j * ld] = w;
        return zabs2(w);
    });
}

// vprev <- v, v <- w / ||w||; block 0 records alpha and the new beta.
__global__ void k_lz_shift(int64_t N, int nl, z_t *V, z_t *Vprev, const z_t *W, int64_t ld,
                           const double *dot_partial, const double *norm_partial, int nb,
                           double *alpha_out, double *beta_out, ChaseScalars *sc) {
    __shared__ double b_s[8];
    if (threadIdx.x < nl) {
        const double nn = sum_partials(norm_partial, nb, nl, threadIdx.x);
        b_s[threadIdx.x] = sqrt(nn);
        if (blockIdx.x == 0 && blockIdx.y == 0) {
            alpha_out[threadIdx.x] = sum_partials(dot_partial, nb, nl, threadIdx.x);
            if (!isfinite(nn)) set_error(sc, DEV_NONFINITE, threadIdx.x);
        }
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < N && j < nl) {
        const double b = b_s[j];
        const double inv = (b > 0.0) ? 1.0 / b : 0.0;
        Vprev[i + j * ld] = V[i + j * ld];
        V[i + j * ld] = zscale(W[i + j * ld], inv);
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < nl) beta_out[threadIdx.x] = b_s[threadIdx.x];
}

}  // namespace

int vec_partial_blocks(int64_t N) {
    int64_t nb = (N + 255) / 256;
    if (nb > 2 * 152) nb = 2 * 152;
    if (nb < 1) nb = 1;
    return (int)nb;
}

cudaError_t launch_col_norms(int64_t N, int nc, const z_t *X, int64_t ldx, double *out,
                             int take_sqrt, double *work, ChaseScalars *sc, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    const int nb = vec_partial_blocks(N);
    k_col_sq<<<nb, kVT, 0, st>>>(N, nc, X, ldx, work);
    bse_count_launches(1);
    k_finish_norms<<<(nc + 127) / 128, 128, 0, st>>>(nb, nc, work, out, take_sqrt, sc);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_col_inv_scale(int64_t N, int nc, z_t *X, int64_t ldx, const double *s,
                                 cudaStream_t st) {
    if (nc <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)nc);
    k_col_inv_scale<<<grid, 256, 0, st>>>(N, nc, X, ldx, s);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_normalize_cols(int64_t N, int nc, z_t *X, int64_t ldx, double *work,
                                  double *norms, ChaseScalars *sc, cudaStream_t st) {
    cudaError_t e = launch_col_norms(N, nc, X, ldx, norms, 1, work, sc, st);
    if (e != cudaSuccess) return e;
    return launch_col_inv_scale(N, nc, X, ldx, norms, st);
}

cudaError_t launch_residuals(int64_t N, int nc, const z_t *HV, int64_t ldhv, const z_t *V,
                             int64_t ldv, const double *theta, double *r, double *work,
                             ChaseScalars *sc, cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    const int nb = vec_partial_blocks(N);
    k_resid<<<nb, kVT, 0, st>>>(N, nc, HV, ldhv, V, ldv, theta, work);
    bse_count_launches(1);
    k_finish_resid<<<(nc + 127) / 128, 128, 0, st>>>(nb, nc, work, r, sc);
    bse_count_launches(1);
    return cudaGetLastError();
}

// The strict upper triangle from the lower one: H(i, j) = conj(H(j, i)) for
// i < j.  One 32 x 32 tile of the upper triangle per CTA (row tile ti <=
// column tile tj), read from its mirror tile and written through shared
// memory, so loads and stores are both coalesced.  A diagonal tile reads all
// of itself before it writes its upper half.
__global__ void __launch_bounds__(256) k_mirror_lower(int64_t N, z_t *H, int64_t ldh) {
    const int ti = blockIdx.x, tj = blockIdx.y;
    if (ti > tj) return;
    __shared__ z_t t[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t i0 = (int64_t)ti * 32, j0 = (int64_t)tj * 32;
    for (int c = ty; c < 32; c += 8) {               // t[c][x] = H(j0 + x, i0 + c)
        const int64_t r = j0 + tx, col = i0 + c;
        if (r < N && col < N) t[c][tx] = H[r + col * ldh];
    }
    __syncthreads();
    for (int c = ty; c < 32; c += 8) {               // H(i0 + x, j0 + c) = conj(t[x][c])
        const int64_t r = i0 + tx, col = j0 + c;
        if (r < N && col < N && r < col) H[r + col * ldh] = zconj(t[tx][c]);
    }
}

cudaError_t launch_mirror_lower(int64_t N, z_t *H, int64_t ldh, cudaStream_t st) {
    if (N <= 1) return cudaSuccess;
    const unsigned T = (unsigned)((N + 31) / 32);
    k_mirror_lower<<<dim3(T, T), dim3(32, 8), 0, st>>>(N, H, ldh);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_copy_cols(int64_t N, int nc, const z_t *in, int64_t ldin, z_t *out,
                             int64_t ldout, const int *perm, cudaStream_t st) {
    if (nc <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)nc);
    k_copy_cols<<<grid, 256, 0, st>>>(N, nc, in, ldin, out, ldout, perm);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_select_cols(int64_t N, int nc, const z_t *A, const z_t *B, int64_t ld,
                               const int *deg, int parity, z_t *out, cudaStream_t st) {
    if (nc <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)nc);
    k_select_cols<<<grid, 256, 0, st>>>(N, nc, A, B, ld, deg, parity, out);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_random_block(uint64_t seed, uint64_t stream, int64_t n, int m, int col0,
                                z_t *V, int64_t ldv, cudaStream_t st) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)m);
    k_random_block<<<grid, 256, 0, st>>>(seed, stream, n, col0, V, ldv);
    bse_count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lanczos_step(int64_t N, int nl, z_t *V, z_t *Vprev, z_t *W, int64_t ld,
                                double *alpha_out, const double *beta_prev, double *beta_out,
                                double *work, ChaseScalars *sc, cudaStream_t st) {
    if (nl <= 0 || nl > 8) return cudaErrorInvalidValue;
    const int nb = vec_partial_blocks(N);
    double *dotp = work, *normp = work + (int64_t)nb * nl;
    k_lz_dot<<<nb, kVT, 0, st>>>(N, nl, V, W, ld, dotp);
    bse_count_launches(1);
    k_lz_update<<<nb, kVT, 0, st>>>(N, nl, V, Vprev, W, ld, dotp, nb, beta_prev, normp);
    bse_count_launches(1);
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)nl);
    k_lz_shift<<<grid, 256, 0, st>>>(N, nl, V, Vprev, W, ld, dotp, normp, nb, alpha_out, beta_out,
                                     sc);
    bse_count_launches(1);
    return cudaGetLastError();
}

namespace {
// Each column's largest-modulus entry (smallest index on ties) is made real
// and positive by a unit phase; one block per column.
__global__ void k_phase_normalize(int64_t N, z_t *X, int64_t ldx) {
    __shared__ double best_v[8];
    __shared__ int64_t best_i[8];
    __shared__ z_t ph_s;
    z_t *x = X + (int64_t)blockIdx.x * ldx;
    double bv = -1.0;
    int64_t bi = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double a = zabs2(x[i]);
        if (a > bv) { bv = a; bi = i; }   // strided scan: first index wins ties
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) { best_v[warp] = bv; best_i[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); w++)
            if (best_v[w] > bv || (best_v[w] == bv && best_i[w] < bi)) { bv = best_v[w]; bi = best_i[w]; }
        const z_t v = x[bi];
        const double a = sqrt(zabs2(v));
        ph_s = (a > 0.0) ? zmk(v.x / a, -v.y / a) : zmk(1.0, 0.0);
    }
    __syncthreads();
    const z_t ph = ph_s;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) x[i] = zmul(x[i], ph);
    __syncthreads();
    if (threadIdx.x == 0) {
        // the pivot becomes exactly real
        const z_t v = x[bi];
        x[bi] = zmk(v.x, 0.0);
    }
}
}  // namespace

cudaError_t launch_phase_normalize(int64_t N, int nc, z_t *X, int64_t ldx, cudaStream_t st) {
    if (nc <= 0 || N <= 0) return cudaSuccess;
    k_phase_normalize<<<nc, 256, 0, st>>>(N, X, ldx);
    bse_count_launches(1);
    return cudaGetLastError();
}
