// Seeded synthetic BSE Hamiltonian of Eq. (1) on the device.
//
// H_{vck, v'c'k'} = (E_ck - E_vk) delta delta delta + 2 vbar - W (Sec. 2,
// Eq. (1)).  The real matrix elements come from DFT data the paper reads
// from disk (Sec. 2, "Read optics" / "Reading/Building"); this generator is
// a seeded stand-in with the same structure:
//   pair index     I(k, v, c) = (k*Nv + v)*Nc + c,   N = Nk*Nv*Nc
//   bands          s(k) = (1 - cos(2 pi k/Nk))/2 on a periodic 1-D k ring
//                  E_c = gap/2 + c + 3 disp s(k) + jitter xi(k, c)
//                  E_v = -gap/2 - v/2 - 2 disp s(k)
//   exchange       2 sum_r a_r(I) conj(a_r(J)), a_r = sqrt(3 x0/N)(u1 + i u2)/sqrt(2)
//   direct         w0 / (d(k,k')^2 + 1/2) e^{i(theta_I - theta_J)} for equal (v, c)
// with u, xi uniform on [-1, 1] and theta uniform on [0, 2 pi) drawn from
// SplitMix64 (Steele, Lea, Flood 2014) keyed by seed ^ (stream << 56) ^ index.
//
// Two kernels: a per-pair table pass (O(N)), then one thread per element.
// An element above the diagonal is computed as the conjugate of its mirror,
// evaluated by the same code, so H is Hermitian bit for bit and every
// column is written with coalesced stores.  HBM traffic: 16 N^2 bytes.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// tables: dE[N], theta[N], a[N*R] (pair-major: a[I*R + r])
__global__ void bse_tables_kernel(uint64_t seed, int Nk, int Nv, int Nc, BseModel md,
                                  double *dE, double *theta, z_t *a) {
    const int64_t N = (int64_t)Nk * Nv * Nc;
    const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= N) return;
    const int c = (int)(I % Nc);
    const int v = (int)((I / Nc) % Nv);
    const int k = (int)(I / ((int64_t)Nc * Nv));
    const double s = (1.0 - cos(kTwoPi * (double)k / (double)Nk)) / 2.0;
    const double xi = 2.0 * unif(seed, 1, (uint64_t)k * Nc + c) - 1.0;
    const double Ec = md.band_gap / 2.0 + c + 3.0 * md.dispersion * s + md.jitter * xi;
    const double Ev = -md.band_gap / 2.0 - 0.5 * v - 2.0 * md.dispersion * s;
    dE[I] = Ec - Ev;
    theta[I] = kTwoPi * unif(seed, 3, (uint64_t)I);
    const double amp = sqrt(3.0 * md.x0 / (double)N) / sqrt(2.0);
    for (int r = 0; r < md.rank_x; r++) {
        const uint64_t idx = 2 * ((uint64_t)md.rank_x * I + r);
        const double u1 = 2.0 * unif(seed, 2, idx) - 1.0;
        const double u2 = 2.0 * unif(seed, 2, idx + 1) - 1.0;
        a[I * md.rank_x + r] = zmk(amp * u1, amp * u2);
    }
}

__device__ __forceinline__ z_t lower_element(int64_t I, int64_t J, int Nk, int nb, BseModel md,
                                             const double *dE, const double *theta, const z_t *a) {
    const int R = md.rank_x;
    z_t x = zmk(0.0, 0.0);
    for (int r = 0; r < R; r++) x = zadd(x, zmul(a[I * R + r], zconj(a[J * R + r])));
    x = zscale(x, 2.0);
    z_t w = zmk(0.0, 0.0);
    if (I % nb == J % nb) {
        int64_t dk = I / nb - J / nb;
        if (dk < 0) dk = -dk;
        if (Nk - dk < dk) dk = Nk - dk;
        const double K = 1.0 / ((double)dk * (double)dk + 0.5);
        const double ph = theta[I] - theta[J];
        double sn, cs;
        sincos(ph, &sn, &cs);
        w = zmk(md.w0 * K * cs, md.w0 * K * sn);
    }
    if (I == J) return zmk(dE[I] + x.x - w.x, 0.0);
    return zsub(x, w);
}

__global__ void bse_matrix_kernel(int Nk, int nb, int64_t N, BseModel md, const double *dE,
                                  const double *theta, const z_t *a, z_t *H, int64_t ldh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int64_t j = blockIdx.y; j < N; j += gridDim.y) {
        z_t h = (i >= j) ? lower_element(i, j, Nk, nb, md, dE, theta, a)
                         : zconj(lower_element(j, i, Nk, nb, md, dE, theta, a));
        H[i + j * ldh] = h;
    }
}

}  // namespace

cudaError_t launch_bse_build(uint64_t seed, int Nk, int Nv, int Nc, const BseModel &md,
                             double *dE, double *theta, z_t *a, z_t *H, int64_t ldh,
                             cudaStream_t st) {
    const int64_t N = (int64_t)Nk * Nv * Nc;
    bse_tables_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(seed, Nk, Nv, Nc, md, dE, theta, a);
    bse_count_launches(1);
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)(N < 65535 ? N : 65535));
    bse_matrix_kernel<<<grid, 256, 0, st>>>(Nk, Nv * Nc, N, md, dE, theta, a, H, ldh);
    bse_count_launches(1);
    return cudaGetLastError();
}
