// One element of the seeded synthetic BSE Hamiltonian (Eq. (1) stand-in),
// shared by the kernel that writes H (gen.cu) and the kernel that writes its
// tensor-core slices without storing H (genslice.cu), so both produce the
// same bits.
//
// The caller stages, for the 32 rows I and 32 columns J of a tile: the
// exchange vectors a_r(I) at ai[r * stride] and a_r(J) at aj[r * stride],
// u_I = e^{i theta_I}, u_J, and dE_I; Kt[d] = 1 / (d^2 + 1/2).
#pragma once
#include "common.cuh"
#include "kernels.h"

// H(I, J) for I >= J: dE_I [I = J] + 2 sum_r a_r(I) conj(a_r(J))
//                     - w0 Kt[d(k_I, k_J)] [b_I = b_J] u_I conj(u_J)
// with k = I / nb, b = I % nb (nb = Nv Nc band pairs), d the ring distance.
__device__ __forceinline__ z_t bse_element(int I, int J, int R, const z_t *ai, const z_t *aj,
                                           int stride, z_t uI, z_t uJ, double dEI, int Nk, int nb,
                                           double w0, const double *Kt) {
    z_t x = zmk(0.0, 0.0);                   // sum_r a_Ir conj(a_Jr)
    for (int r = 0; r < R; r++) {
        const z_t ar = ai[r * stride], as = aj[r * stride];
        x.x = fma(ar.x, as.x, x.x);
        x.x = fma(ar.y, as.y, x.x);
        x.y = fma(ar.y, as.x, x.y);
        x.y = fma(-ar.x, as.y, x.y);
    }
    x = zscale(x, 2.0);
    z_t w = zmk(0.0, 0.0);
    if (I % nb == J % nb) {
        int dk = I / nb - J / nb;
        if (dk < 0) dk = -dk;
        if (Nk - dk < dk) dk = Nk - dk;
        w = zscale(zmul(uI, zconj(uJ)), w0 * Kt[dk]);
    }
    return (I == J) ? zmk(dEI + x.x - w.x, 0.0) : zsub(x, w);
}
