/*
 * bsechase: ChASE (Chebyshev-accelerated subspace iteration) for the lowest
 * eigenpairs of a dense complex Hermitian Bethe-Salpeter (exciton)
 * Hamiltonian, on one GB300 GPU (sm_103a).
 *
 * The problem is the one of arXiv 2006.08498: the eigenproblem of the BSE
 * Hamiltonian of Eq. (1) (Sec. 2), for the lowest part of the spectrum with
 * eigenvectors (Sec. 2, the optical response needs the eigenvectors), with
 * the solver's search-space parameters nev and nex (Sec. 3, and the nex
 * study of the Supplement).  The solver's phases are those of the
 * Supplement's ChASE timing breakdown: Lanczos, Filter, QR, Rayleigh-Ritz,
 * Resid.
 *
 * Conventions for every entry point:
 *  - Matrices are column-major: element (i, j) at p[i + j*ld], ld >= rows.
 *  - Complex numbers are interleaved (re, im) doubles (C99 double complex,
 *    torch.complex128).  A row-major Hermitian H passed as-is is conj(H):
 *    same eigenvalues, conjugated eigenvectors.
 *  - "d_" pointers are CUDA device pointers on the context's device; "h_"
 *    pointers and plain double* outputs are host memory.
 *  - The caller owns every buffer it passes; the library owns its workspace
 *    (allocated in the context, grown on demand, freed by destroy) and never
 *    frees caller memory.
 *  - All device work is issued on the context's stream.  Entry points
 *    return after their results are complete (host outputs written).
 *  - Every call returns a status (bse_status); no exception crosses the
 *    ABI.  bsechase_last_error() describes the last failure of a context.
 *  - Threads: a context is used by one host thread at a time; separate
 *    contexts (on the same or on different devices) may be used from
 *    separate threads concurrently.  The library's one-time kernel set-up
 *    (launch attributes, cluster checks) is done once per device under a
 *    lock.  The request server runs its own threads, one context each.
 */
#ifndef BSECHASE_H
#define BSECHASE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsechase_ctx bsechase_ctx;

typedef enum {
    BSE_OK = 0,
    BSE_EINVAL = -1,     /* invalid argument (size, pointer, parameter)       */
    BSE_ENOMEM = -2,     /* device workspace could not be allocated           */
    BSE_ENOCONV = -3,    /* max_iter reached; converged pairs are returned and
                            the residual of every other pair is +inf          */
    BSE_ENONFINITE = -4, /* NaN/Inf met (in H or in a reduction), or a
                            Cholesky factorisation failed                     */
    BSE_ETIMEOUT = -5,   /* a bounded wait expired                            */
    BSE_ECUDA = -6,      /* a CUDA runtime call failed                        */
    BSE_EBUSY = -7       /* the request is still pending                      */
} bse_status;

typedef enum {
    CHASE_FP64 = 0,       /* FP64 accuracy.  Products with H (Lanczos, filter,
                             Rayleigh-Ritz) run on the BF16 tensor cores as an
                             Ozaki-scheme emulation: 6 slices of 8 bits per
                             operand, exact integer accumulation of the
                             slice diagonals 2..5 per K chunk of 64, FP32 for
                             diagonals 6..7 (normwise error ~1e-12 relative
                             to ||H|| ||Y||).  QR, reduced eig,
                             residuals and locking in native FP64.          */
    CHASE_MIXED_FP32 = 1, /* filter products at FP32-level accuracy on the
                             tensor cores (first 4 slices: 32 bits relative to
                             the row/column maximum, 10 slice pairs) while
                             every unlocked residual exceeds 1e-6, then on 5
                             slices (15 pairs) while every one exceeds 1e-8,
                             then FP64-accurate filter sweeps; Lanczos, QR,
                             Rayleigh-Ritz and residuals as in CHASE_FP64.
                             In single-phase entry points it selects the
                             FP32-level product.                             */
    CHASE_MIXED_BF16X3 = 2, /* accepted and run as CHASE_MIXED_FP32, the
                             closest built mode: its filter products are
                             BF16 split products too, with four slices,
                             because three 8-bit slices (about 24 bits per
                             operand, products accurate to ~1e-5 relative to
                             ||H|| ||Y|| on these matrices) cannot carry the
                             residuals to the point where the FP64-accurate
                             sweeps take over.  Results are bit for bit those
                             of CHASE_MIXED_FP32.                             */
    CHASE_FP64_DFMA = 3   /* every product in native FP64 (DFMA)            */
} chase_precision;

/* Parameters of the synthetic Eq. (1) Hamiltonian (energies in eV).
 * NULL selects the defaults {2.0, 0.3, 0.5, 0.01, 1.0, 8}. */
typedef struct {
    double band_gap;    /* E_c(k=0,c=0) - E_v(k=0,v=0) without jitter         */
    double w0;          /* strength of the screened direct term W             */
    double x0;          /* strength of the exchange term 2 vbar               */
    double jitter;      /* amplitude of the seeded conduction-band jitter     */
    double dispersion;  /* scale of the cosine band dispersion                */
    int rank_x;         /* rank of the exchange term (0..64)                  */
} bse_model;

/* Solver options; NULL selects the defaults. */
typedef struct {
    int deg_init;        /* first-iteration filter degree (default 20)       */
    int max_iter;        /* iteration limit (default 50)                      */
    int lanczos_steps;   /* steps per Lanczos run (default 25, <= 64)         */
    int lanczos_vecs;    /* independent Lanczos runs (default 4, <= 8)        */
    uint64_t seed;       /* seed of the Lanczos and start vectors (default 0) */
    const void *d_V0;    /* optional warm start: N x n_v0 device block        */
    int64_t ldv0;
    int n_v0;            /* 0 = none; at most nev + nex columns are used      */
    int degree_group;    /* 0 (default): the per-vector degrees of Eq. (S1).
                            > 0: before each filter the degrees (ascending) are
                            taken in groups of this many columns from the
                            highest down and raised to the group's largest.
                            A filter product costs the same for any column
                            count within one tile of the tensor-core kernel
                            (48 columns), so 48 filters some columns further
                            at no cost; never lowers a degree.  No counterpart
                            in the paper. */
    double nex_damping;  /* 0 (default): nex fixed.  > 0: the nex tuner (the
                            Supplement's nex study, Tables S8/S9: the damping
                            1/rho_nev of Eq. (S1) with gamma = lambda_nev sets
                            the convergence rate, and a larger nex lowers it).
                            After each Rayleigh-Ritz from the second on, the
                            damping is evaluated with gamma = the nev-th Ritz
                            value and alpha = the largest; once two consecutive
                            values differ by at most 0.02 and the value exceeds
                            nex_damping, nex grows once to min(max(2 nex,
                            nex + 8), min(N, 512) - nev).  The new columns are
                            the seeded start block's next columns. */
    int half_storage;    /* 0 (default): the tensor-core slices of all of H
                            (24 N^2 bytes).  1: of its lower triangle only
                            (12 N^2 bytes), the strict upper triangle never
                            read (H is Hermitian; the paper's reader holds one
                            triangle, Sec. 3): rows are scaled symmetrically,
                            H = T S T with t_i = sqrt(max_k |H_ik|), so that
                            one exponent serves S's rows and its columns, and
                            the product reads each stored tile of S both
                            ways.  The products keep the normwise accuracy
                            of full storage; row by row it is relative to
                            sqrt(max_k |H_ik| max |H|) rather than to the
                            row's own maximum, so the small rows of a
                            strongly graded H are less accurate.  Tensor-core
                            precisions only (BSE_EINVAL otherwise).  With chase_solve_bse the slices are
                            generated, so H's whole footprint is 12 N^2
                            bytes. */
} chase_opts;

/* Per-solve statistics (times in milliseconds, CUDA events on the stream). */
typedef struct {
    int iters;              /* subspace iterations                            */
    int locked;             /* pairs converged                                */
    int64_t matvecs;        /* H*vector products: filter + RR + Lanczos       */
    int64_t filter_matvecs; /* filter products only                          */
    double ms_lanczos, ms_filter, ms_qr, ms_rr, ms_resid, ms_total;
    double filter_tflops;   /* 8 N^2 filter_matvecs / filter time             */
    double norm_est;        /* ||H|| estimate (Lanczos)                       */
    double alpha, beta, lower; /* final damped interval and filter lower point */
    int64_t kernel_launches;   /* CUDA kernels this solve launched            */
    int64_t filter_launches;   /* filter matrix-product launches              */
    int64_t filter_matvecs_low; /* filter products at FP32-level accuracy
                                   (4 slices; CHASE_MIXED_FP32)               */
    /* The tensor-core product kernel alone (precisions FP64 and MIXED_FP32),
     * timed with CUDA events around each launch on the solver's stream:    */
    double tc_kernel_ms;        /* summed launch durations                    */
    int64_t tc_kernel_launches; /* launches timed                             */
    double tc_kernel_tflops;    /* executed BF16 tensor flops (8 per complex  */
                                /* multiply-add per slice pair) / duration    */
    int nex_used;               /* nex at the end (differs from the argument
                                   when the nex tuner grew it)                */
    int64_t filter_matvecs_mid; /* filter products on 5 slices
                                   (CHASE_MIXED_FP32)                         */
    int64_t h2d_bytes, d2h_bytes; /* host<->device bytes copied by
                                   chase_solve_host (0 for the other calls)   */
    double ms_h2d;              /* chase_solve_host: copy of H's lower
                                   triangle and its mirroring on the device   */
} chase_stats;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = a stream owned by the context). */
int bsechase_create(bsechase_ctx **ctx, int device, void *cuda_stream);
/* Free the context's workspace and stream (if owned).  NULL is ignored. */
void bsechase_destroy(bsechase_ctx *ctx);
/* Static description of a status code. */
const char *bsechase_strerror(int status);
/* Description of the last failure in `ctx` (empty string if none). */
const char *bsechase_last_error(const bsechase_ctx *ctx);

/* Time limit, in seconds (0 < seconds <= 60, default 2), of every bounded
 * wait inside the context's tensor-core kernels (a wait for a copy, an MMA or
 * a drained accumulator).  When a wait runs out, the kernel stops issuing
 * work, waits for the copies and MMAs it already issued, releases its tensor
 * memory and returns; the call then fails with BSE_ETIMEOUT and the context
 * stays usable.  A short limit makes that path run on purpose (failure
 * detection tests).  The paper has no counterpart.  Errors: BSE_EINVAL. */
int bsechase_set_wait_limit(bsechase_ctx *ctx, double seconds);

/* Page-locked host memory for the host-buffer calls (chase_solve_host):
 * *p receives `bytes` of host memory allocated by the CUDA runtime, which the
 * copy engines read at the host link's full rate for as long as it lives.
 * Free it with bsechase_host_free.  Errors: BSE_EINVAL (p NULL or bytes 0),
 * BSE_ENOMEM. */
int bsechase_host_alloc(void **p, size_t bytes);
/* Free memory from bsechase_host_alloc (NULL is ignored).  Errors: BSE_ECUDA. */
int bsechase_host_free(void *p);

/* Dimension N = Nk * Nv * Nc of the BSE Hamiltonian (Sec. 2: the pair index
 * runs over valence bands, conduction bands and k-points); -1 if invalid. */
int64_t bse_dim(int Nk, int Nv, int Nc);

/* Fill d_H (N x N complex128, column-major, leading dimension ldh >= N)
 * with the seeded synthetic BSE Hamiltonian of Eq. (1):
 *   H_IJ = dE_I delta_IJ + 2 sum_r a_r(I) conj(a_r(J))
 *          - w0 [v=v', c=c'] e^{i(theta_I - theta_J)} / (d(k,k')^2 + 1/2),
 * I = (k Nv + v) Nc + c, dE = E_c(k) - E_v(k) from cosine bands with jitter,
 * d the distance on a periodic ring of Nk k-points, a_r, theta and the
 * jitter drawn from SplitMix64 keyed by `seed`.  H is Hermitian bit for bit.
 * Errors: BSE_EINVAL (sizes <= 0, N > 2^31, ldh < N, rank_x outside 0..64,
 * NULL d_H), BSE_ECUDA. */
int bse_build_hamiltonian(bsechase_ctx *ctx, uint64_t seed, int Nk, int Nv, int Nc,
                          const bse_model *model, void *d_H, int64_t ldh);

/* Lowest nev eigenpairs of the Hermitian d_H (N x N complex128,
 * column-major, ldh >= N) by ChASE (Sec. 3; Supplement, ChASE breakdown).
 * Search space m = nev + nex (1 <= nev, 0 <= nex, m <= min(N, 512)).
 * Converged means ||H v - lambda v||_2 / ||H||_est <= tol, ||H||_est from
 * the Lanczos estimate; deg_max (>= 2) caps the per-vector filter degree.
 * Outputs: h_evals[nev] ascending; d_evecs (N x nev complex128, ld = ldz >=
 * N) orthonormal, each column's largest-modulus entry (smallest index on
 * ties) real and positive; h_resid[nev]; stats (nullable).
 * d_H is read only (with chase_opts.half_storage, only its lower triangle).
 * Errors: BSE_EINVAL, BSE_ENOMEM, BSE_ENOCONV (outputs
 * filled, unconverged residuals +inf), BSE_ENONFINITE, BSE_ECUDA. */
int chase_solve(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, int nev, int nex,
                double tol, int deg_max, int precision, const chase_opts *opts, double *h_evals,
                void *d_evecs, int64_t ldz, double *h_resid, chase_stats *stats);

/* As chase_solve for the synthetic Hamiltonian of bse_build_hamiltonian
 * (same seed, Nk, Nv, Nc, model), without storing it: its elements are
 * generated straight into the tensor-core slices of H, so the N x N
 * complex128 matrix (16 N^2 bytes) never exists and the device memory the
 * solve needs drops from 40 N^2 to 24 N^2 bytes plus workspace, 12 N^2 with
 * chase_opts.half_storage (Sec. 3's
 * filter works on H only through its products).  The slices, and so every
 * result, are bit for bit those of bse_build_hamiltonian + chase_solve.
 * Tensor-core precisions only (CHASE_FP64, CHASE_MIXED_FP32, value 2);
 * CHASE_FP64_DFMA needs the stored H: BSE_EINVAL.  Other errors as
 * chase_solve. */
int chase_solve_bse(bsechase_ctx *ctx, uint64_t seed, int Nk, int Nv, int Nc,
                    const bse_model *model, int nev, int nex, double tol, int deg_max,
                    int precision, const chase_opts *opts, double *h_evals, void *d_evecs,
                    int64_t ldz, double *h_resid, chase_stats *stats);

/* As chase_solve with every matrix in HOST memory: the lower triangle of h_H
 * (N x N, diagonal included) is copied to a context-owned device buffer, the
 * upper triangle is taken as its conjugate transpose (H is Hermitian; the
 * paper's reader likewise holds one triangle, Sec. 3), and the eigenvectors
 * are copied back into h_evecs (N x nev, ld = ldz).  The strict upper triangle
 * of h_H is never read.  Host buffers should be page-locked
 * (bsechase_host_alloc) for full transfer speed; stats, when given, also
 * report the bytes copied each way and the copy's time.  Same errors as
 * chase_solve. */
int chase_solve_host(bsechase_ctx *ctx, const void *h_H, int64_t N, int64_t ldh, int nev,
                     int nex, double tol, int deg_max, int precision, const chase_opts *opts,
                     double *h_evals, void *h_evecs, int64_t ldz, double *h_resid,
                     chase_stats *stats);

/* ---- single phases, on caller device buffers (the steps chase_solve runs) */

/* Lanczos spectral estimate (Supplement, "Lanczos" item): `runs` Lanczos
 * runs of `steps` steps from SplitMix64 start vectors (seed, stream 4).
 * out[4] (host) = {beta (upper bound of lambda_N), mu_1 (estimate of
 * lambda_1), mu_m (estimate of lambda_m), ||H|| estimate}. */
int chase_lanczos(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, int m,
                  int steps, int runs, uint64_t seed, int precision, double *out);

/* Chebyshev filter (Sec. 3; Supplement, "Filter" item): column j of d_V
 * (N x m, ldv) is replaced by p_{d_j}(H) v_j, p_d(x) = T_d((x-c)/e) /
 * T_d((lower-c)/e), via the scaled three-term recurrence.  h_deg[m] (host)
 * must be ascending, each >= 1.  Returns the number of H*vector products
 * in *matvecs (nullable). */
int chase_filter(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, void *d_V,
                 int64_t ldv, int m, const int *h_deg, double lower, double c, double e,
                 int precision, int64_t *matvecs);

/* QR phase (Supplement, "QR" item): d_V (N x m) becomes an orthonormal
 * basis of span(d_V) projected off span(d_L) (d_L: N x k orthonormal, may
 * be NULL with k = 0): two projections, column scaling, shifted Cholesky QR
 * and two Cholesky QR passes each after a projection. */
int chase_qr(bsechase_ctx *ctx, const void *d_L, int64_t ldl, int k, void *d_V, int64_t ldv,
             int64_t N, int m);

/* Rayleigh-Ritz (Supplement, "RR" item) for orthonormal d_Q (N x m):
 * h_theta[m] ascending Ritz values; d_V = Q Y and d_HV = H Q Y (N x m,
 * ld = N); h_resid[m] = ||HV_j - theta_j V_j|| / norm (nullable). */
int chase_rayleigh_ritz(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh,
                        const void *d_Q, int64_t ldq, int m, int precision, double *h_theta,
                        void *d_V, void *d_HV, double norm, double *h_resid);

/* Gram product of the QR and Rayleigh-Ritz phases (Supplement, "QR" and
 * "RR" items): d_G (m1 x m2, ldg >= m1) = A^H B for A: K x m1 (lda), B: K x m2
 * (ldb), 1 <= m1, m2 <= 512.  Split over K with a fixed partition and a
 * fixed-order sum (run-to-run deterministic); partial sums live in the
 * context's workspace. */
int chase_gram(bsechase_ctx *ctx, const void *d_A, int64_t lda, const void *d_B, int64_t ldb,
               int64_t K, int m1, int m2, void *d_G, int64_t ldg);

/* Allocation-free Gram product, for callers that cannot allocate device
 * memory (their memory manager owns the device, they cannot afford the
 * allocator's synchronisation, or they cannot create a context, which
 * allocates workspace).  The paper has no counterpart: it is a service entry
 * point.  Same result as chase_gram (G = A^H B, m1 x m2, ldg >= m1, for A: K x
 * m1, B: K x m2) computed on the current device and on `cuda_stream` (NULL =
 * the default stream); the call returns once the work is enqueued.  The
 * split-K partial sums live in a fixed 4 MiB device array inside the library
 * (held by every GPU that loads it, until exit), so no memory is allocated;
 * m1, m2 > 512 is rejected with BSE_EINVAL.  The first call on a device looks
 * up that array's address; make it before any stream capture begins.  Every
 * call shares the array: calls whose work overlaps on the GPU race and must be
 * serialised by the caller.  Errors: BSE_EINVAL, BSE_ECUDA. */
int chase_gram_noalloc(const void *d_A, int64_t lda, const void *d_B, int64_t ldb, int64_t K,
                       int m1, int m2, void *d_G, int64_t ldg, void *cuda_stream);

/* The filter's matrix product alone: d_C = H d_Y (d_Y: N x n, ldy; d_C: N x n,
 * ldc; 1 <= n <= 512) at the given precision (Sec. 3: the filter is a
 * repeated HEMM).  d_C must not overlap d_H or d_Y. */
int chase_hemm(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, const void *d_Y,
               int64_t ldy, int n, void *d_C, int64_t ldc, int precision);
/* As chase_hemm on the tensor cores with the first `slices` 8-bit slices of
 * each operand (4, 5 or 6; slice pairs p + q <= slices + 1): 6 is CHASE_FP64's
 * product, 4 the FP32-level product of CHASE_MIXED_FP32, 5 the intermediate
 * level that mode uses between them (about 40 bits per operand relative to
 * its row or column maximum).  half_storage = 1: the product on the slices
 * of H's lower triangle (chase_opts.half_storage; the strict upper triangle
 * of d_H is not read).  Other values: BSE_EINVAL. */
int chase_hemm_slices(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh,
                      const void *d_Y, int64_t ldy, int n, void *d_C, int64_t ldc, int slices,
                      int half_storage);

/* ---- request server (continuous batching of many solves on one GPU) ------
 * The paper's BSE workflow solves sequences of related eigenproblems (k-mesh
 * and energy-cutoff convergence tests, Sec. 2 and Sec. 4); the server runs a
 * stream of such solves.  Requests are admitted in FIFO order when a slot is
 * free and their memory estimate fits the HBM budget; each slot has its own
 * stream, so admitted requests run concurrently; results (eigenvalues,
 * residuals, stats, latency stamps) stay with the server until released, and
 * eigenvectors stay on the device (LRU-evicted under the budget) so later
 * requests can warm-start from them. */

typedef struct {
    uint64_t seed;           /* synthetic Hamiltonian: bse_build_hamiltonian   */
    int Nk, Nv, Nc;
    int use_model;           /* 0: default model parameters                    */
    bse_model model;
    int nev, nex;            /* as chase_solve                                 */
    double tol;
    int deg_max, precision;
    uint64_t warm_ticket;    /* 0, or a ticket whose eigenvectors (same N) start
                                this solve if that request has finished       */
    int degree_group;        /* as chase_opts.degree_group (0: Eq. (S1))       */
    double nex_damping;      /* as chase_opts.nex_damping (0: nex fixed)       */
    const void *d_H;         /* NULL: the synthetic Hamiltonian above.  Else the
                                caller's N x N Hermitian matrix on the server's
                                device (N = Nk Nv Nc, column-major, ld = ldh),
                                read by the solve and not copied: the caller
                                keeps it unchanged until the request finishes */
    int64_t ldh;
    int half_storage;        /* as chase_opts.half_storage                     */
    int h_free;              /* 1: the synthetic Hamiltonian is not stored (as
                                chase_solve_bse; tensor-core precisions, d_H
                                NULL): 16 N^2 bytes less in the request's
                                budget estimate                               */
} chase_request;

typedef struct {
    int status;              /* the solve's status (as chase_solve)           */
    int has_evecs;           /* eigenvectors resident (chase_server_evecs)     */
    int64_t N;
    int nev;
    const double *evals;     /* nev, ascending; valid until released          */
    const double *resid;     /* nev                                          */
    chase_stats stats;
    double t_submit, t_start, t_end;  /* seconds, steady clock                */
} chase_result;

/* Start a server on ctx's device: max_slots (1..64) concurrent solves within
 * hbm_budget_bytes of admitted memory.  One server per context. */
int chase_server_create(bsechase_ctx *ctx, size_t hbm_budget_bytes, int max_slots);
/* Queue a request; *ticket identifies it.  BSE_EINVAL (bad request), BSE_ENOMEM
 * (its estimate exceeds the whole budget). */
int chase_server_submit(bsechase_ctx *ctx, const chase_request *req, uint64_t *ticket);
/* BSE_EBUSY while pending; BSE_OK and *out filled when finished. */
int chase_server_poll(bsechase_ctx *ctx, uint64_t ticket, chase_result *out);
/* Block up to timeout_s seconds; BSE_ETIMEOUT if still pending. */
int chase_server_wait(bsechase_ctx *ctx, uint64_t ticket, double timeout_s, chase_result *out);
/* Copy a finished request's eigenvectors (N x nev) to d_out (device or host
 * memory, leading dimension ld >= N). */
int chase_server_evecs(bsechase_ctx *ctx, uint64_t ticket, void *d_out, int64_t ld);
/* Cancel a queued request, or drop a finished one's results and eigenvectors
 * (BSE_EBUSY while it runs or while a queued warm start depends on it). */
int chase_server_release(bsechase_ctx *ctx, uint64_t ticket);
/* Product batching (off by default): with enabled = 1 the tensor-core
 * products that the running solves submit within window_s of each other, or
 * as soon as every running solve has submitted one, run in one launch of the
 * persistent product kernel, each with the same work units and arithmetic as
 * alone (results are unchanged, bit for bit).  With enabled = 0 every product
 * is launched on its own slot's stream, and the slots' kernels overlap on the
 * device by stream concurrency alone; on the serving mix of mixed sizes this
 * measured faster (the window delays launches, and a shared launch waits for
 * its slowest member's operands).  Only while no request is queued or running
 * (BSE_EBUSY otherwise).  No counterpart in the paper. */
int chase_server_batching(bsechase_ctx *ctx, int enabled, double window_s);
/* Launches the batcher made, products they carried, and the most products
 * in one launch. */
int chase_server_batch_stats(bsechase_ctx *ctx, int64_t *launches, int64_t *products,
                             int *max_products);
/* Admitted bytes (running + resident), queued and running requests. */
int chase_server_info(bsechase_ctx *ctx, size_t *held_bytes, int *queued, int *running);
/* Stop the workers (waits for running solves) and free everything. */
int chase_server_destroy(bsechase_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* BSECHASE_H */
