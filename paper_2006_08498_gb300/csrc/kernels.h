// Internal launch interface between the host driver and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

struct BseModel {
    double band_gap, w0, x0, jitter, dispersion;
    int rank_x;
};

// ---- generator (gen.cu)
// Tables (device scratch): dE[N], u[N] = e^{i theta}, a[N * rank_x] and
// Kt[Nk / 2 + 1] = 1 / (d^2 + 1/2).  launch_bse_tables writes the tables
// alone; launch_bse_build writes them and then H.
cudaError_t launch_bse_tables(uint64_t seed, int Nk, int Nv, int Nc, const BseModel &md,
                              double *dE, z_t *u, z_t *a, double *Kt, cudaStream_t st);
cudaError_t launch_bse_build(uint64_t seed, int Nk, int Nv, int Nc, const BseModel &md,
                             double *dE, z_t *u, z_t *a, double *Kt, z_t *H, int64_t ldh,
                             cudaStream_t st);

// ---- dense products (zgemm.cu)
enum GemmMode { GEMM_PLAIN = 0, GEMM_SUB = 1, GEMM_CHEB = 2 };
struct GemmEpi {
    int mode;
    double s1, c, s2;      // CHEB: C = s1 (AB - c B[i,j]) - s2 Yp[i,j]
    const z_t *Yp;         // CHEB: previous iterate (may alias C); null when s2 == 0
    int64_t ldyp;
    const z_t *D;          // SUB: C = D - AB (may alias C)
    int64_t ldd;
    int b_upper;           // B is upper triangular: B[k, j] = 0 for k > j (skipped)
};
// C[M x n] = epi(A[M x K] B[K x n]), all column-major FP64 complex.
cudaError_t launch_zgemm_nn(int64_t M, int64_t n, int64_t K, const z_t *A, int64_t lda,
                            const z_t *B, int64_t ldb, z_t *C, int64_t ldc, const GemmEpi &ep,
                            cudaStream_t st);
// G[m1 x m2] = A^H B (+ shift on the diagonal), A: K x m1, B: K x m2; split-K
// partial sums in `work` (>= zgemm_cn_work_elems(..) elements), reduced in a
// fixed order so the result is deterministic.
int64_t zgemm_cn_work_elems(int64_t m1, int64_t m2, int64_t K);
// The split count is reduced if ns * m1 * m2 would exceed work_elems.
cudaError_t launch_zgemm_cn(int64_t m1, int64_t m2, int64_t K, const z_t *A, int64_t lda,
                            const z_t *B, int64_t ldb, z_t *G, int64_t ldg, double shift,
                            int hermitize, z_t *work, int64_t work_elems, cudaStream_t st);

// ---- FP64-accurate products on the BF16 tensor cores (ozaki.cu)
// H sliced once per solve: A slices (ozaki_a_bytes), row exponents E
// (padded length), and the TMA descriptor of the slices.
// Time limit of each bounded mbarrier wait inside the tensor-core kernel
// (nanoseconds of %globaltimer); on expiry the kernel winds down and reports
// DEV_TIMEOUT.
constexpr uint64_t kDefaultWaitNs = 2000000000ull;

// Accuracy levels of the tensor-core product: the first S slices of 8 bits
// of each operand (relative to its row or column maximum), slice pairs
// p + q <= S + 1.  OZ_S6: FP64 accuracy (21 pairs); OZ_S4: FP32 level
// (10 pairs, products ~3e-8 relative to ||H|| ||Y||); OZ_S5: 15 pairs, 256
// times more accurate than OZ_S4.
enum OzLevel { OZ_S6 = 0, OZ_S4 = 1, OZ_S5 = 2 };
inline int oz_pairs(int level) { return level == OZ_S4 ? 10 : level == OZ_S5 ? 15 : 21; }

// The slices of H, prepared once per solve.  Full storage: all Np x Np
// elements, one exponent per row.  Half storage (tri): the lower-triangle
// tiles of the symmetrically scaled S = D H D, D = diag(s_i), s_i = 1 / t_i,
// t_i = sqrt(max_k |H_ik|) (1 + 2^-20), so that S is Hermitian with |S_ik|
// < 1 and one exponent (0) serves every row; the product reads the upper
// tiles as the conjugate transposes of the stored ones and computes
// H Y = T (S (T Y)), T = diag(t_i).
struct OzakiH {
    int64_t N = 0, Np = 0;
    void *A = nullptr;
    int *E = nullptr;
    uint64_t wait_ns = kDefaultWaitNs;
    bool tri = false;
    double *t = nullptr, *s = nullptr;   // tri: t_i and s_i = 1 / t_i (Np each)
    alignas(64) unsigned char tmap[128];
    alignas(64) unsigned char tmap2[128];   // tri: 64-row boxes of the stored tiles
};
int64_t ozaki_padded(int64_t N);
size_t ozaki_a_bytes(int64_t N);
// Half storage: the 128 x 64 tiles of the lower triangle, T (T + 1) per
// part, T = Np / 128.
size_t ozaki_a_bytes_tri(int64_t N);
size_t ozaki_b_bytes(int64_t N, int m);
// workspace for split-K partial products of up to m columns
size_t ozaki_partial_bytes(int64_t N, int m);

// General FP64-accurate products on the tensor cores (same kernel and
// slicing as the product with H): C (M x n) = out(op(A) B), op(A) = A
// (M x K) or A^H (ah = 1: A is K x M); B is K x n.  out: OZ_PLAIN C = op(A)B,
// OZ_SUB C = D - op(A)B (D may alias C), OZ_GRAM (M = n) C = op(A)B, its
// Hermitian part if hermitize, plus shift on the diagonal.  Workspace:
// slices of op(A) (ozaki_gen_a_bytes) with M-long exponents E, slices of B
// (ozaki_gen_b_bytes) with n-long exponents F, raw partials (24 bytes) of n M
// complex values per split.
enum { OZ_PLAIN = 0, OZ_SUB = 1, OZ_GRAM = 2 };
struct OzGemmWork {
    void *A = nullptr;
    size_t a_bytes = 0;
    int *E = nullptr;
    int64_t e_len = 0;
    void *B = nullptr;
    size_t b_bytes = 0;
    int *F = nullptr;
    int64_t f_len = 0;
    z_t *P = nullptr;
    size_t p_bytes = 0;
    uint64_t wait_ns = kDefaultWaitNs;
};
size_t ozaki_gen_a_bytes(int64_t M, int64_t K);
size_t ozaki_gen_b_bytes(int64_t K, int n);
cudaError_t ozaki_gemm(int64_t M, int n, int64_t K, const z_t *A, int64_t lda, int ah,
                       const z_t *B, int64_t ldb, int mode, const z_t *D, int64_t ldd,
                       double shift, int hermitize, z_t *C, int64_t ldc, const OzGemmWork &w,
                       ChaseScalars *sc, int sms, cudaStream_t st);
// The slices of the synthetic Hamiltonian generated from the generator's
// tables (launch_bse_tables) without storing H; oh->A and oh->E must hold
// ozaki_a_bytes(N) and Np ints.  The values are those bse_build_hamiltonian
// writes, bit for bit.
// With tri: half storage (the layout of ozaki_prepare_h_tri; oh->t and oh->s
// hold Np entries each), bit for bit ozaki_prepare_h_tri on the built H.
cudaError_t ozaki_prepare_bse(int Nk, int Nv, int Nc, const BseModel &md, const double *dE,
                              const z_t *u, const z_t *a, const double *Kt, bool tri, OzakiH *oh,
                              ChaseScalars *sc, cudaStream_t st);
// Non-finite entries of H (or of a product's operand) set DEV_NONFINITE in sc.
cudaError_t ozaki_prepare_h(int64_t N, const z_t *H, int64_t ldh, OzakiH *oh, ChaseScalars *sc,
                            cudaStream_t st);
// Half storage from the lower triangle of H (the strict upper triangle is
// never read); oh->A >= ozaki_a_bytes_tri(N), oh->E, oh->t and oh->s hold Np
// entries each.
cudaError_t ozaki_prepare_h_tri(int64_t N, const z_t *H, int64_t ldh, OzakiH *oh,
                                ChaseScalars *sc, cudaStream_t st);
// C[N x n] = epi(H Y), Y: N x n (ld ldy); bslices >= ozaki_b_bytes(N, n),
// F >= padded n ints.  GEMM_PLAIN or GEMM_CHEB epilogues (C may alias Yp).
// level (OzLevel): how many slices of each operand take part.
// K is split across CTAs (raw int64 + FP32 partials in `partials`, summed in a fixed
// order) when that fills the `sms` multiprocessors better.  When ev0/ev1
// are given they are recorded on `st` just before and after the
// tensor-core kernel itself (not the slicing or the split-K sum).
// With a batcher, the tensor-core kernel is launched by the batcher together
// with other threads' products (ev0/ev1 are then not recorded).
struct OzBatcher;
cudaError_t ozaki_zgemm(const OzakiH &oh, int n, const z_t *Y, int64_t ldy, z_t *C, int64_t ldc,
                        const GemmEpi &ep, void *bslices, int *F, ChaseScalars *sc, int level,
                        z_t *partials, size_t partial_bytes, int sms, cudaStream_t st,
                        cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                        OzBatcher *batcher = nullptr);
// Product batcher shared by the solver threads of a request server: products
// submitted within window_s of each other (or as soon as every active solver
// has submitted one) run in one launch of the tensor-core kernel.
OzBatcher *ozb_create(int device, int sms, double window_s);
void ozb_destroy(OzBatcher *b);
void ozb_set_active(OzBatcher *b, int n);   // solvers that may submit
void ozb_set_window(OzBatcher *b, double window_s);
void ozb_counts(OzBatcher *b, int64_t *launches, int64_t *jobs, int *max_jobs);

// ---- vector kernels (vec.cu)
int vec_partial_blocks(int64_t N);
// out[j] = sum_i |X[i,j]|^2 (sqrt if take_sqrt) for j < nc; partials in work
cudaError_t launch_col_norms(int64_t N, int nc, const z_t *X, int64_t ldx, double *out,
                             int take_sqrt, double *work, ChaseScalars *sc, cudaStream_t st);
// X[:, j] *= 1/s[j]
cudaError_t launch_col_inv_scale(int64_t N, int nc, z_t *X, int64_t ldx, const double *s,
                                 cudaStream_t st);
// r[j] = ||HV[:,j] - theta[j] V[:,j]|| / sc->norm_est
cudaError_t launch_residuals(int64_t N, int nc, const z_t *HV, int64_t ldhv, const z_t *V,
                             int64_t ldv, const double *theta, double *r, double *work,
                             ChaseScalars *sc, cudaStream_t st);
// out[:, j] = in[:, perm ? perm[j] : j]
// H(i, j) = conj(H(j, i)) for i < j (N x N, column-major): the Hermitian
// matrix whose lower triangle H holds.
cudaError_t launch_mirror_lower(int64_t N, z_t *H, int64_t ldh, cudaStream_t st);
cudaError_t launch_copy_cols(int64_t N, int nc, const z_t *in, int64_t ldin, z_t *out,
                             int64_t ldout, const int *perm, cudaStream_t st);
// Seeded complex block (2u-1) + i(2u'-1) from SplitMix64, as in the generator
cudaError_t launch_random_block(uint64_t seed, uint64_t stream, int64_t n, int m, int col0,
                                z_t *V, int64_t ldv, cudaStream_t st);
// Lanczos: per column l: a_l = Re(v_l^H w_l) (dots), then
// w_l -= a_l v_l + b_l v_prev_l (b_l = beta_prev[l]), b'_l = ||w_l||,
// v_prev <- v, v <- w / b'; a_l -> alpha_out[l], b'_l -> beta_out[l].
cudaError_t launch_lanczos_step(int64_t N, int nl, z_t *V, z_t *Vprev, z_t *W, int64_t ld,
                                double *alpha_out, const double *beta_prev, double *beta_out,
                                double *work, ChaseScalars *sc, cudaStream_t st);
// Unit phase making each column's largest-modulus entry real positive.
cudaError_t launch_phase_normalize(int64_t N, int nc, z_t *X, int64_t ldx, cudaStream_t st);
cudaError_t launch_normalize_cols(int64_t N, int nc, z_t *X, int64_t ldx, double *work,
                                  double *norms, ChaseScalars *sc, cudaStream_t st);
// out[:, j] = sel[j] ? B[:, j] : A[:, j]   (gather of filter results)
cudaError_t launch_select_cols(int64_t N, int nc, const z_t *A, const z_t *B, int64_t ld,
                               const int *deg, int parity, z_t *out, cudaStream_t st);

// ---- single-CTA small dense kernels (small.cu)
// In-place Cholesky G = R^H R (upper R, n x n); failure recorded in sc.
cudaError_t launch_cholesky(int n, z_t *G, int64_t ld, ChaseScalars *sc, cudaStream_t st);
// X = R^{-1} for upper-triangular R (n x n)
cudaError_t launch_trinv(int n, const z_t *R, int64_t ldr, z_t *X, int64_t ldx, cudaStream_t st);
// Eigen-decomposition of Hermitian A (n x n, may be overwritten): ascending w, vectors Y.
size_t heev_work_bytes(int n);
cudaError_t launch_heev(int n, z_t *A, int64_t lda, double *w, z_t *Y, int64_t ldy, void *work,
                        ChaseScalars *sc, cudaStream_t st);
// Lanczos estimates from the n_runs tridiagonals (alpha[k*nl + l], beta[k*nl + l]).
cudaError_t launch_lanczos_finalize(int k, int nl, int64_t N, int m, const double *alpha,
                                    const double *beta, ChaseScalars *sc, cudaStream_t st);
// Locking, interval update, degrees and degree sort after a Rayleigh-Ritz step.
// Inputs theta/resid of the m_act active pairs (ascending theta).  Outputs:
// sc->new_locked / locked / alpha / lower, deg[0..m_act-nl) (ascending) and
// perm (the Ritz index of each unlocked column after sorting).
cudaError_t launch_chase_update(int m_act, int nev, double tol, int deg_max,
                                const double *theta, const double *resid, int *deg, int *perm,
                                ChaseScalars *sc, cudaStream_t st);
