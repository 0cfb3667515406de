/* A plain C user of the library: builds the synthetic Eq. (1) Hamiltonian
 * on the device, solves for its lowest eigenpairs through chase_solve and
 * through chase_solve_bse (H never stored, half storage), and prints the
 * eigenvalues.  Used by tests/test_gpu_c_abi.py (compiled with a C compiler
 * against include/bsechase.h, the CUDA runtime and libbsechase.so).
 *
 * usage: c_abi_solve Nk nev nex  ->  "status iters" lines and nev values */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "bsechase.h"

static int check(bsechase_ctx *ctx, int rc, const char *what) {
    if (rc != BSE_OK) {
        fprintf(stderr, "%s: %s (%s)\n", what, bsechase_strerror(rc),
                ctx ? bsechase_last_error(ctx) : "");
        return 1;
    }
    return 0;
}

int main(int argc, char **argv) {
    if (argc != 4) return 2;
    const int Nk = atoi(argv[1]), nev = atoi(argv[2]), nex = atoi(argv[3]);
    const int64_t N = bse_dim(Nk, 4, 4);
    if (N < 1) return 2;
    bsechase_ctx *ctx = NULL;
    if (check(NULL, bsechase_create(&ctx, 0, NULL), "create")) return 1;
    void *dH = NULL, *dZ = NULL;
    if (cudaMalloc(&dH, (size_t)(16 * N * N)) != cudaSuccess ||
        cudaMalloc(&dZ, (size_t)(16 * N * nev)) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    double *ev = (double *)malloc(sizeof(double) * (size_t)nev);
    double *res = (double *)malloc(sizeof(double) * (size_t)nev);
    chase_stats st;
    int rc = 0;
    rc |= check(ctx, bse_build_hamiltonian(ctx, 0, Nk, 4, 4, NULL, dH, N), "build");
    rc |= check(ctx, chase_solve(ctx, dH, N, N, nev, nex, 1e-10, 36, CHASE_FP64, NULL, ev, dZ, N,
                                 res, &st), "solve");
    if (rc) return 1;
    printf("solve %d %d\n", BSE_OK, st.iters);
    for (int j = 0; j < nev; j++) printf("%.17e %.3e\n", ev[j], res[j]);
    cudaFree(dH);
    chase_opts o = {0};
    o.half_storage = 1;
    rc |= check(ctx, chase_solve_bse(ctx, 0, Nk, 4, 4, NULL, nev, nex, 1e-10, 36, CHASE_FP64, &o,
                                     ev, dZ, N, res, &st), "solve_bse");
    if (rc) return 1;
    printf("solve_bse %d %d\n", BSE_OK, st.iters);
    for (int j = 0; j < nev; j++) printf("%.17e %.3e\n", ev[j], res[j]);
    cudaFree(dZ);
    free(ev);
    free(res);
    bsechase_destroy(ctx);
    return 0;
}
