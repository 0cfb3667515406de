// Host driver and C ABI of the ChASE solver (include/bsechase.h).
//
// The iteration follows the phases of the Supplement's ChASE breakdown
// (Lanczos once, then Filter -> QR -> Rayleigh-Ritz -> Resid/lock until
// nev pairs are locked).  Every phase runs in the kernels of gen.cu,
// zgemm.cu, vec.cu and small.cu on the context's stream; the host only
// sequences launches and reads back, once per iteration, the scalars and
// the per-vector degrees that size the next filter's launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/bsechase.h"
#include "context.h"
#include "kernels.h"

namespace {

constexpr int kMaxM = 512;
constexpr double kU = 0x1.0p-53;
constexpr double kKappaMax = 1e12;             // cap on the filter's amplification
// Mixed precision: the filter runs on the first four slices (FP32 level)
// while every unlocked pair's residual is above kMixedSwitch, on five while
// every one is above kMixedSwitch5, then FP64-accurate sweeps close the
// solve.  Each level's residual floor lies about a decade below its switch
// point (four slices: near 1e-7; five: 256 times lower).
constexpr double kMixedSwitch = 1e-6;
constexpr double kMixedSwitch5 = 1e-8;
constexpr int64_t kCnWork = (int64_t)1 << 20;   // split-K partials (complex elements)
constexpr int64_t kHostCopyCols = 256;           // columns per copy of the lower triangle

}  // namespace

int fail(bsechase_ctx *c, int code, const char *fmt, const char *detail) {
    char buf[512];
    snprintf(buf, sizeof buf, fmt, detail);
    c->err = buf;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return fail(ctx, BSE_ECUDA, "CUDA error: %s", cudaGetErrorString(e_)); \
    } while (0)

// Grow a workspace buffer; allocations are stream-ordered on the context's
// stream, so growing one context's workspace never synchronises the device
// (other contexts keep running).
int ensure(bsechase_ctx *ctx, DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes) return BSE_OK;
    if (b.p) cudaFreeAsync(b.p, ctx->st);
    b.p = nullptr;
    b.bytes = 0;
    if (bytes == 0) return BSE_OK;
    if (cudaMallocAsync(&b.p, bytes, ctx->st) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, BSE_ENOMEM, "cannot allocate %s of device workspace",
                    std::to_string(bytes).c_str());
    }
    b.bytes = bytes;
    return BSE_OK;
}

void release_workspace(bsechase_ctx *ctx) {
    DevBuf *bufs[] = {&ctx->V,  &ctx->B1,      &ctx->B2,   &ctx->B3,  &ctx->G,      &ctx->R,
                      &ctx->Ri, &ctx->Yr,      &ctx->heev, &ctx->small_d, &ctx->ints, &ctx->part,
                      &ctx->lz, &ctx->tables, &ctx->Hdev, &ctx->Zdev, &ctx->ozA, &ctx->ozE,
                      &ctx->ozB, &ctx->ozF, &ctx->ozP, &ctx->ozGA, &ctx->ozGE, &ctx->ozT};
    for (DevBuf *b : bufs) {
        if (b->p) cudaFreeAsync(b->p, ctx->st);
        b->p = nullptr;
        b->bytes = 0;
    }
    ctx->wsN = 0;
    ctx->wsM = 0;
}

void harvest_kernel_times(bsechase_ctx *ctx) {
    for (size_t i = 0; i + 1 < ctx->kev_used; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->kev[i], ctx->kev[i + 1]) == cudaSuccess) {
            ctx->k_ms += ms;
            ctx->k_flops += ctx->kev_flops[i / 2];
            ctx->k_launches++;
        } else {
            cudaGetLastError();
        }
    }
    ctx->kev_used = 0;
    ctx->kev_flops.clear();
}

namespace {

// Small-array layout inside small_d (doubles) and ints.
struct Small {
    double *theta, *resid, *norms, *lz_alpha, *lz_beta, *lam, *res;
    int *deg, *perm, *order;
};

Small small_layout(bsechase_ctx *ctx, int m) {
    Small s;
    double *d = (double *)ctx->small_d.p;
    s.theta = d;
    s.resid = d + kMaxM;
    s.norms = d + 2 * kMaxM;
    s.lz_alpha = d + 3 * kMaxM;          // 64 x 8
    s.lz_beta = d + 3 * kMaxM + 512;     // (64 + 1) x 8: row 0 = zeros
    s.lam = d + 3 * kMaxM + 1088;
    s.res = d + 4 * kMaxM + 1088;
    int *ip = (int *)ctx->ints.p;
    s.deg = ip;
    s.perm = ip + kMaxM;
    s.order = ip + 2 * kMaxM;
    (void)m;
    return s;
}

int ensure_workspace(bsechase_ctx *ctx, int64_t N, int m) {
    int rc;
    const size_t blk = (size_t)N * m * sizeof(z_t);
    if ((rc = ensure(ctx, ctx->V, blk))) return rc;
    if ((rc = ensure(ctx, ctx->B1, blk))) return rc;
    if ((rc = ensure(ctx, ctx->B2, blk))) return rc;
    if ((rc = ensure(ctx, ctx->B3, blk))) return rc;
    const size_t sq = (size_t)kMaxM * kMaxM * sizeof(z_t);
    if ((rc = ensure(ctx, ctx->G, sq))) return rc;
    if ((rc = ensure(ctx, ctx->R, sq))) return rc;
    if ((rc = ensure(ctx, ctx->Ri, sq))) return rc;
    if ((rc = ensure(ctx, ctx->Yr, sq))) return rc;
    if ((rc = ensure(ctx, ctx->heev, heev_work_bytes(kMaxM)))) return rc;
    if ((rc = ensure(ctx, ctx->small_d, (size_t)(6 * kMaxM + 2048) * sizeof(double)))) return rc;
    if ((rc = ensure(ctx, ctx->ints, (size_t)4 * kMaxM * sizeof(int)))) return rc;
    const size_t cn = (size_t)kCnWork * sizeof(z_t);
    const size_t vp = (size_t)vec_partial_blocks(N) * kMaxM * 2 * sizeof(double);
    if ((rc = ensure(ctx, ctx->part, std::max(cn, vp)))) return rc;
    if ((rc = ensure(ctx, ctx->lz, (size_t)N * 8 * 3 * sizeof(z_t)))) return rc;
    ctx->wsN = N;
    ctx->wsM = m;
    return BSE_OK;
}

int check_device_error(bsechase_ctx *ctx) {
    const int e = ctx->hsc->error;
    if (e == DEV_OK) return BSE_OK;
    const std::string where = std::to_string(ctx->hsc->error_where);
    switch (e) {
        case DEV_CHOL_FAIL:
            return fail(ctx, BSE_ENONFINITE, "Cholesky factorisation failed at column %s",
                        where.c_str());
        case DEV_EIG_NOCONV:
            return fail(ctx, BSE_ENONFINITE, "reduced eigensolver did not converge (%s)",
                        where.c_str());
        case DEV_NONFINITE:
            return fail(ctx, BSE_ENONFINITE, "non-finite value in a reduction (column %s)",
                        where.c_str());
        case DEV_TIMEOUT:
            return fail(ctx, BSE_ETIMEOUT, "a bounded wait in a tensor-core kernel expired (CTA %s)",
                        where.c_str());
        default:
            return fail(ctx, BSE_ECUDA, "device error %s", std::to_string(e).c_str());
    }
}

int sync_scalars(bsechase_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->hsc, ctx->sc, sizeof(ChaseScalars), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    harvest_kernel_times(ctx);
    return check_device_error(ctx);
}

// ------------------------------------------------------- the operator H
// Every product with H goes through Hop: native FP64 (zgemm.cu) or the
// FP64-accurate tensor-core emulation (ozaki.cu), fixed per solve.
struct Hop {
    const z_t *H;
    int64_t N, ldh;
    bool tc;         // tensor-core emulation
    int level = OZ_S6;   // slices of the tensor-core product (mixed precision filter)
    const BseSource *bse = nullptr;   // H not stored: its slices from the generator
    bool tri = false;    // half storage of the slices (lower triangle of H only)
};

int hop_prepare(bsechase_ctx *ctx, Hop &op, int max_cols) {
    if (!op.tc) return BSE_OK;
    int rc;
    const int64_t Np = ozaki_padded(op.N);
    if ((rc = ensure(ctx, ctx->ozA, op.tri ? ozaki_a_bytes_tri(op.N) : ozaki_a_bytes(op.N))))
        return rc;
    if (op.tri && (rc = ensure(ctx, ctx->ozT, (size_t)2 * Np * sizeof(double)))) return rc;
    if ((rc = ensure(ctx, ctx->ozE, (size_t)Np * sizeof(int)))) return rc;
    const int mc = std::max(max_cols, 32);
    if ((rc = ensure(ctx, ctx->ozB, ozaki_b_bytes(op.N, mc)))) return rc;
    if ((rc = ensure(ctx, ctx->ozF, (size_t)(mc + 64) * sizeof(int)))) return rc;
    const size_t pbytes = ozaki_partial_bytes(op.N, mc);
    if ((rc = ensure(ctx, ctx->ozP, pbytes))) return rc;
    // general products of QR and Rayleigh-Ritz: op(A) is m x N (A^H) or N x m
    const size_t gab = std::max(ozaki_gen_a_bytes(mc, op.N), ozaki_gen_a_bytes(op.N, mc));
    if ((rc = ensure(ctx, ctx->ozGA, gab))) return rc;
    if ((rc = ensure(ctx, ctx->ozGE, (size_t)(Np + 512) * sizeof(int)))) return rc;
    ctx->oh.A = ctx->ozA.p;
    ctx->oh.E = (int *)ctx->ozE.p;
    ctx->oh.wait_ns = ctx->wait_ns;
    ctx->oh.t = (double *)ctx->ozT.p;
    ctx->oh.s = ctx->oh.t ? ctx->oh.t + Np : nullptr;
    if (op.bse)
        CK(ozaki_prepare_bse(op.bse->Nk, op.bse->Nv, op.bse->Nc, op.bse->md, op.bse->dE, op.bse->u,
                             op.bse->a, op.bse->Kt, op.tri, &ctx->oh, ctx->sc, ctx->st));
    else if (op.tri)
        CK(ozaki_prepare_h_tri(op.N, op.H, op.ldh, &ctx->oh, ctx->sc, ctx->st));
    else
        CK(ozaki_prepare_h(op.N, op.H, op.ldh, &ctx->oh, ctx->sc, ctx->st));
    return BSE_OK;
}

// Two timing events for the next tensor-core launch (null when no event
// can be created: the launch then goes untimed).
void kernel_events(bsechase_ctx *ctx, double flops, cudaEvent_t *e0, cudaEvent_t *e1) {
    *e0 = *e1 = nullptr;
    while (ctx->kev.size() < ctx->kev_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        ctx->kev.push_back(e);
    }
    *e0 = ctx->kev[ctx->kev_used];
    *e1 = ctx->kev[ctx->kev_used + 1];
    ctx->kev_used += 2;
    ctx->kev_flops.resize(ctx->kev_used / 2);
    ctx->kev_flops.back() = flops;
}

// C[N x n] = epi(H Y)
int hop_apply(bsechase_ctx *ctx, const Hop &op, int n, const z_t *Y, int64_t ldy, z_t *C,
              int64_t ldc, const GemmEpi &ep) {
    if (op.tc) {
        // tensor flops: 8 real flops per complex multiply-add for each of
        // the 21 (FP64), 15 or 10 (FP32-level) slice pairs
        const double pairs = oz_pairs(op.level);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        // a batched launch holds other solvers' products: not timed per product
        if (!ctx->batcher)
            kernel_events(ctx, 8.0 * pairs * (double)op.N * (double)op.N * n, &e0, &e1);
        CK(ozaki_zgemm(ctx->oh, n, Y, ldy, C, ldc, ep, ctx->ozB.p, (int *)ctx->ozF.p, ctx->sc,
                       op.level, (z_t *)ctx->ozP.p, ctx->ozP.bytes, ctx->sms, ctx->st, e0,
                       e1, ctx->batcher));
    } else
        CK(launch_zgemm_nn(op.N, n, op.N, op.H, op.ldh, Y, ldy, C, ldc, ep, ctx->st));
    return BSE_OK;
}

}  // namespace

bool precision_uses_tc(int precision) {
    return precision == CHASE_FP64 || precision == CHASE_MIXED_FP32;
}

bool precision_valid(int precision) {
    return precision == CHASE_FP64 || precision == CHASE_MIXED_FP32 ||
           precision == CHASE_MIXED_BF16X3 || precision == CHASE_FP64_DFMA;
}
// The mode a valid precision value runs: CHASE_MIXED_BF16X3 runs as
// CHASE_MIXED_FP32 (see the header), every other value as itself.
int precision_mode(int precision) {
    return precision == CHASE_MIXED_BF16X3 ? CHASE_MIXED_FP32 : precision;
}

namespace {

// ---------------------------------------------------------------- phases

// Lanczos estimate; results land in ctx->sc (beta, mu_1, mu_m, norm_est,
// alpha = mu_m, lower = mu_1).
int phase_lanczos(bsechase_ctx *ctx, const Hop &op, int m, int steps, int runs, uint64_t seed) {
    const int64_t N = op.N;
    if (steps < 1 || steps > 64 || runs < 1 || runs > 8) return fail(ctx, BSE_EINVAL, "bad Lanczos size%s");
    Small s = small_layout(ctx, m);
    z_t *Vl = (z_t *)ctx->lz.p, *Vp = Vl + N * 8, *W = Vp + N * 8;
    const int k = (int)std::min<int64_t>(steps, N);
    CK(launch_random_block(seed, 4, N, runs, 0, Vl, N, ctx->st));
    CK(launch_normalize_cols(N, runs, Vl, N, (double *)ctx->part.p, s.norms, ctx->sc, ctx->st));
    CK(cudaMemsetAsync(Vp, 0, (size_t)N * runs * sizeof(z_t), ctx->st));
    CK(cudaMemsetAsync(s.lz_beta, 0, 8 * sizeof(double), ctx->st));
    GemmEpi plain{};
    for (int j = 0; j < k; j++) {
        int rc;
        if ((rc = hop_apply(ctx, op, runs, Vl, N, W, N, plain))) return rc;
        // beta_{j-1} (zeros before the first step) -> beta_j
        const double *bprev = (j == 0) ? s.lz_beta : s.lz_beta + 8 + (j - 1) * runs;
        CK(launch_lanczos_step(N, runs, Vl, Vp, W, N, s.lz_alpha + j * runs, bprev,
                               s.lz_beta + 8 + j * runs, (double *)ctx->part.p, ctx->sc, ctx->st));
    }
    // beta history for the finaliser: row j of lz_beta + 8 holds beta_j
    CK(launch_lanczos_finalize(k, runs, N, m, s.lz_alpha, s.lz_beta + 8, ctx->sc, ctx->st));
    return BSE_OK;
}

// Filter columns V[:, 0..m) (degrees ascending, host copy h_deg, device copy
// d_deg) in place; B1 is the second buffer of the recurrence.
int phase_filter(bsechase_ctx *ctx, const Hop &op, z_t *V, int64_t ldv, int m, const int *h_deg,
                 const int *d_deg, double lower, double c, double e, int64_t *matvecs,
                 int64_t *launches = nullptr) {
    if (m <= 0) return BSE_OK;
    const int64_t N = op.N;
    int rc;
    z_t *B1 = (z_t *)ctx->B1.p;
    const int64_t ldb = N;
    const double sigma1 = e / (lower - c);
    GemmEpi ep{};
    ep.mode = GEMM_CHEB;
    ep.s1 = sigma1 / e;
    ep.c = c;
    ep.s2 = 0.0;
    ep.Yp = nullptr;
    // Y_1 = (sigma_1/e)(H Y_0 - c Y_0) into B1; Y_t lives in V (t even) or B1 (t odd)
    if ((rc = hop_apply(ctx, op, m, V, ldv, B1, ldb, ep))) return rc;
    int64_t mv = m;
    double sigma = sigma1;
    const int dmax = h_deg[m - 1];
    for (int t = 1; t < dmax; t++) {
        int s = 0;
        while (s < m && h_deg[s] <= t) s++;
        const double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
        z_t *cur = (t & 1) ? B1 : V;
        z_t *prv = (t & 1) ? V : B1;
        const int64_t ldc = (t & 1) ? ldb : ldv, ldp = (t & 1) ? ldv : ldb;
        ep.s1 = 2.0 * sigma_new / e;
        ep.s2 = sigma * sigma_new;
        ep.Yp = prv + s * ldp;
        ep.ldyp = ldp;
        if ((rc = hop_apply(ctx, op, m - s, cur + s * ldc, ldc, prv + s * ldp, ldp, ep))) return rc;
        mv += m - s;
        sigma = sigma_new;
    }
    // column j's result Y_{d_j} is in B1 when d_j is odd
    if (ldv != ldb) return fail(ctx, BSE_EINVAL, "filter block needs ld = N%s");
    CK(launch_select_cols(N, m, V, B1, ldv, d_deg, 1, V, ctx->st));
    if (matvecs) *matvecs = mv;
    if (launches) *launches += dmax;
    return BSE_OK;
}

// V -= L (L^H V)
// The N x m products of QR and Rayleigh-Ritz: on the tensor cores with
// FP64-level accuracy when the solve's products with H are (ctx->gen_tc),
// else native FP64.  The operands here are orthonormal or unit-norm
// columns, so the per-row/per-column scaling of the slices keeps the error
// at FP64 rounding level.
struct GenTcScope {
    bsechase_ctx *c;
    GenTcScope(bsechase_ctx *ctx, bool on) : c(ctx) { c->gen_tc = on; }
    ~GenTcScope() { c->gen_tc = false; }
};

OzGemmWork gen_work(bsechase_ctx *ctx) {
    OzGemmWork w;
    w.A = ctx->ozGA.p;
    w.a_bytes = ctx->ozGA.bytes;
    w.E = (int *)ctx->ozGE.p;
    w.e_len = (int64_t)(ctx->ozGE.bytes / sizeof(int));
    w.B = ctx->ozB.p;
    w.b_bytes = ctx->ozB.bytes;
    w.F = (int *)ctx->ozF.p;
    w.f_len = (int64_t)(ctx->ozF.bytes / sizeof(int));
    w.P = (z_t *)ctx->ozP.p;
    w.p_bytes = ctx->ozP.bytes;
    w.wait_ns = ctx->wait_ns;
    return w;
}

// G (m1 x m2) = A^H B (+ shift on the diagonal, Hermitian part if hermitize)
int gemm_cn(bsechase_ctx *ctx, int64_t m1, int64_t m2, int64_t K, const z_t *A, int64_t lda,
            const z_t *B, int64_t ldb, z_t *G, int64_t ldg, double shift, int hermitize) {
    if (ctx->gen_tc) {
        const int mode = (m1 == m2 && (hermitize || shift != 0.0)) ? OZ_GRAM : OZ_PLAIN;
        CK(ozaki_gemm(m1, (int)m2, K, A, lda, 1, B, ldb, mode, nullptr, 0, shift, hermitize, G, ldg,
                      gen_work(ctx), ctx->sc, ctx->sms, ctx->st));
    } else {
        CK(launch_zgemm_cn(m1, m2, K, A, lda, B, ldb, G, ldg, shift, hermitize,
                           (z_t *)ctx->part.p, kCnWork, ctx->st));
    }
    return BSE_OK;
}

// C (M x n) = A B, or D - A B with sub (D may alias C)
int gemm_nn(bsechase_ctx *ctx, int64_t M, int64_t n, int64_t K, const z_t *A, int64_t lda,
            const z_t *B, int64_t ldb, z_t *C, int64_t ldc, const z_t *D, int64_t ldd,
            bool b_upper) {
    if (ctx->gen_tc) {
        CK(ozaki_gemm(M, (int)n, K, A, lda, 0, B, ldb, D ? OZ_SUB : OZ_PLAIN, D, ldd, 0.0, 0, C,
                      ldc, gen_work(ctx), ctx->sc, ctx->sms, ctx->st));
    } else {
        GemmEpi ep{};
        if (D) {
            ep.mode = GEMM_SUB;
            ep.D = D;
            ep.ldd = ldd;
        }
        ep.b_upper = b_upper ? 1 : 0;
        CK(launch_zgemm_nn(M, n, K, A, lda, B, ldb, C, ldc, ep, ctx->st));
    }
    return BSE_OK;
}

int project(bsechase_ctx *ctx, const z_t *L, int64_t ldl, int k, z_t *V, int64_t ldv, int64_t N,
            int m) {
    if (k <= 0) return BSE_OK;
    z_t *X = (z_t *)ctx->R.p;
    int rc;
    if ((rc = gemm_cn(ctx, k, m, N, L, ldl, V, ldv, X, k, 0.0, 0))) return rc;
    return gemm_nn(ctx, N, m, k, L, ldl, X, k, V, ldv, V, ldv, false);
}

// one Cholesky QR pass: G = V^H V + shift I = R^H R, V <- V R^{-1}
int cholqr_pass(bsechase_ctx *ctx, z_t *V, int64_t ldv, int64_t N, int m, double shift) {
    z_t *G = (z_t *)ctx->G.p, *Ri = (z_t *)ctx->Ri.p, *B1 = (z_t *)ctx->B1.p;
    int rc;
    if ((rc = gemm_cn(ctx, m, m, N, V, ldv, V, ldv, G, m, shift, 1))) return rc;
    CK(launch_cholesky(m, G, m, ctx->sc, ctx->st));
    CK(launch_trinv(m, G, m, Ri, m, ctx->st));
    // R^{-1} is upper triangular
    if ((rc = gemm_nn(ctx, N, m, m, V, ldv, Ri, m, B1, N, nullptr, 0, true))) return rc;
    CK(launch_copy_cols(N, m, B1, N, V, ldv, nullptr, ctx->st));
    return BSE_OK;
}

int phase_qr(bsechase_ctx *ctx, const z_t *L, int64_t ldl, int k, z_t *V, int64_t ldv, int64_t N,
             int m) {
    int rc;
    if (m <= 0) return BSE_OK;
    Small s = small_layout(ctx, m);
    if ((rc = project(ctx, L, ldl, k, V, ldv, N, m))) return rc;
    if ((rc = project(ctx, L, ldl, k, V, ldv, N, m))) return rc;
    CK(launch_normalize_cols(N, m, V, ldv, (double *)ctx->part.p, s.norms, ctx->sc, ctx->st));
    // columns have unit norm, so ||V||_F^2 = m
    const double shift = 11.0 * ((double)N * m + (double)m * (m + 1)) * kU * (double)m;
    if ((rc = cholqr_pass(ctx, V, ldv, N, m, shift))) return rc;
    for (int pass = 0; pass < 2; pass++) {
        if ((rc = project(ctx, L, ldl, k, V, ldv, N, m))) return rc;
        if ((rc = cholqr_pass(ctx, V, ldv, N, m, 0.0))) return rc;
    }
    return BSE_OK;
}

// Rayleigh-Ritz: theta (device), Vout = Q Y (ld N), HVout = H Q Y (ld N)
int phase_rr(bsechase_ctx *ctx, const Hop &op, const z_t *Q, int64_t ldq, int m, double *theta,
             z_t *Vout, z_t *HVout) {
    const int64_t N = op.N;
    z_t *W = (z_t *)ctx->B1.p, *G = (z_t *)ctx->G.p, *Yr = (z_t *)ctx->Yr.p;
    GemmEpi plain{};
    int rc;
    if ((rc = hop_apply(ctx, op, m, Q, ldq, W, N, plain))) return rc;
    if ((rc = gemm_cn(ctx, m, m, N, Q, ldq, W, N, G, m, 0.0, 1))) return rc;
    CK(launch_heev(m, G, m, theta, Yr, m, ctx->heev.p, ctx->sc, ctx->st));
    if ((rc = gemm_nn(ctx, N, m, m, Q, ldq, Yr, m, Vout, N, nullptr, 0, false))) return rc;
    return gemm_nn(ctx, N, m, m, W, N, Yr, m, HVout, N, nullptr, 0, false);
}

struct Timer {
    bsechase_ctx *ctx;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    void mark(int i) {
        if (ctx->ev_ok) cudaEventRecord(ctx->ev[i], ctx->st);
    }
    void add(int phase, int a, int b) {
        float ms = 0.f;
        if (ctx->ev_ok && cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]) == cudaSuccess)
            acc[phase] += ms;
    }
};

int validate_solve(bsechase_ctx *ctx, const void *H, int64_t N, int64_t ldh, int nev, int nex,
                   double tol, int deg_max, int precision, int64_t ldz) {
    if (!ctx) return BSE_EINVAL;
    if (!H) return fail(ctx, BSE_EINVAL, "H is NULL%s");
    if (N < 1 || ldh < N || ldz < N) return fail(ctx, BSE_EINVAL, "bad N or leading dimension%s");
    if (nev < 1 || nex < 0 || (int64_t)nev + nex > N || nev + nex > kMaxM)
        return fail(ctx, BSE_EINVAL, "need 1 <= nev, 0 <= nex, nev + nex <= min(N, 512)%s");
    if (!(tol > 0.0) || deg_max < 2) return fail(ctx, BSE_EINVAL, "need tol > 0 and deg_max >= 2%s");
    if (!precision_valid(precision)) return fail(ctx, BSE_EINVAL, "unsupported precision%s");
    return BSE_OK;
}

}  // namespace

namespace {

// 1/rho of Eq. (S1) for gamma with the damped interval [alpha, beta]
double damping_of(double gamma, double alpha, double beta) {
    const double c = (alpha + beta) / 2.0, e = (beta - alpha) / 2.0;
    const double t = (gamma - c) / e;
    if (fabs(t) <= 1.0) return 1.0;
    return 1.0 / (fabs(t) + sqrt(t * t - 1.0));
}

// the larger nex of the nex tuner: doubled (at least 8 more), nev + nex <=
// min(N, 512)
int grown_nex(int nex, int nev, int64_t N) {
    const int top = (int)std::min<int64_t>(N, kMaxM) - nev;
    return std::min(std::max(2 * nex, nex + 8), top);
}

constexpr double kNexSettled = 0.02;   // consecutive dampings this close: settled

}  // namespace

int solve_device(bsechase_ctx *ctx, const z_t *H, int64_t N, int64_t ldh, int nev, int nex,
                 double tol, int deg_max, int precision, const chase_opts *opts, double *h_evals,
                 z_t *d_evecs, int64_t ldz, double *h_resid, chase_stats *stats,
                 const BseSource *bse) {
    int rc;
    int m = nev + nex;
    chase_opts o{};
    o.deg_init = 20;
    o.max_iter = 50;
    o.lanczos_steps = 25;
    o.lanczos_vecs = 4;
    o.seed = 0;
    if (opts) {
        if (opts->deg_init > 0) o.deg_init = opts->deg_init;
        if (opts->max_iter > 0) o.max_iter = opts->max_iter;
        if (opts->lanczos_steps > 0) o.lanczos_steps = opts->lanczos_steps;
        if (opts->lanczos_vecs > 0) o.lanczos_vecs = opts->lanczos_vecs;
        o.seed = opts->seed;
        o.d_V0 = opts->d_V0;
        o.ldv0 = opts->ldv0;
        o.n_v0 = opts->n_v0;
        o.degree_group = opts->degree_group;
        o.nex_damping = opts->nex_damping;
        o.half_storage = opts->half_storage;
    }
    if (o.d_V0 && (o.n_v0 < 0 || o.ldv0 < N)) return fail(ctx, BSE_EINVAL, "bad warm-start block%s");
    if (o.degree_group < 0) return fail(ctx, BSE_EINVAL, "degree_group must be >= 0%s");
    if (!(o.nex_damping >= 0.0 && o.nex_damping < 1.0))
        return fail(ctx, BSE_EINVAL, "nex_damping must be in [0, 1)%s");
    if (o.half_storage != 0 && (o.half_storage != 1 || !precision_uses_tc(precision)))
        return fail(ctx, BSE_EINVAL, "half_storage = 1 needs a tensor-core precision%s");
    const bool tuner = o.nex_damping > 0.0;
    // the workspace holds the largest search space the tuner may grow to
    const int m_cap = tuner ? nev + std::max(nex, grown_nex(nex, nev, N)) : m;
    if ((rc = ensure_workspace(ctx, N, m_cap))) return rc;
    Small s = small_layout(ctx, m);
    z_t *V = (z_t *)ctx->V.p, *B2 = (z_t *)ctx->B2.p, *B3 = (z_t *)ctx->B3.p;
    Timer tm{ctx};
    const int64_t launches0 = bse_launch_count();
    ctx->kev_used = 0;
    ctx->kev_flops.clear();
    ctx->k_ms = ctx->k_flops = 0.0;
    ctx->k_launches = 0;
    tm.mark(0);
    CK(cudaMemsetAsync(ctx->sc, 0, sizeof(ChaseScalars), ctx->st));
    Hop op{H, N, ldh, precision_uses_tc(precision)};
    op.bse = bse;
    op.tri = o.half_storage == 1;
    if ((rc = hop_prepare(ctx, op, m_cap))) return rc;
    GenTcScope gen_scope(ctx, op.tc);
    if ((rc = phase_lanczos(ctx, op, m, o.lanczos_steps, o.lanczos_vecs, o.seed))) return rc;
    tm.mark(1);
    int64_t matvecs = (int64_t)std::min<int64_t>(o.lanczos_steps, N) * o.lanczos_vecs;
    int64_t filter_mv = 0, filter_launches = 0, filter_mv_low = 0, filter_mv_mid = 0;
    // start block: seeded columns, the first n_v0 replaced by the warm start
    CK(launch_random_block(o.seed, 5, N, m, 0, V, N, ctx->st));
    if (o.d_V0 && o.n_v0 > 0)
        CK(launch_copy_cols(N, std::min(o.n_v0, m), (const z_t *)o.d_V0, o.ldv0, V, N, nullptr,
                            ctx->st));
    if ((rc = sync_scalars(ctx))) return rc;
    tm.add(0, 0, 1);
    double alpha = ctx->hsc->alpha, beta = ctx->hsc->beta, lower = ctx->hsc->lower;
    const double norm_est = ctx->hsc->norm_est;
    int d0 = std::min(o.deg_init + (o.deg_init & 1), deg_max);
    std::vector<int> hdeg(m, d0);
    std::vector<double> lam(m, 0.0), res(m, INFINITY), th(m), rr(m);
    std::vector<int> perm(m);
    int locked = 0, it = 0;
    bool converged = false;
    double damp_prev = -1.0;
    bool grown = false;
    while (it < o.max_iter) {
        it++;
        const int ma = m - locked;
        const int locked0 = locked;
        const double c = (alpha + beta) / 2.0, e = (beta - alpha) / 2.0;
        z_t *Va = V + (int64_t)locked * N;
        // cap the degrees so the filtered block stays numerically full rank:
        // its condition number is about |T_d((lower - c)/e)| <= kKappaMax
        const double tl = fabs((lower - c) / e);
        if (tl > 1.0) {
            int cap = (int)floor(acosh(kKappaMax) / acosh(tl));
            cap -= cap & 1;
            if (cap < 2) cap = 2;
            for (int j = 0; j < ma; j++) hdeg[j] = std::min(hdeg[j], cap);
        }
        // optional degree groups: with the degrees ascending, groups of
        // o.degree_group columns from the highest down take the group's
        // largest degree (a filter step costs the same for any column count
        // within one tile of the product kernel)
        if (o.degree_group > 0) {
            for (int hi = ma; hi > 0;) {
                const int lo = std::max(0, hi - o.degree_group);
                for (int j = lo; j < hi; j++) hdeg[j] = hdeg[hi - 1];
                hi = lo;
            }
        }
        CK(cudaMemcpyAsync(s.deg, hdeg.data(), ma * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
        tm.mark(2);
        int64_t mv = 0;
        Hop fop = op;
        if (precision == CHASE_MIXED_FP32) {
            double rmin = INFINITY;
            for (int j = locked; j < m; j++) rmin = std::min(rmin, res[j]);
            fop.level = rmin > kMixedSwitch ? OZ_S4 : rmin > kMixedSwitch5 ? OZ_S5 : OZ_S6;
        }
        if ((rc = phase_filter(ctx, fop, Va, N, ma, hdeg.data(), s.deg, lower, c, e, &mv,
                               &filter_launches)))
            return rc;
        filter_mv += mv;
        if (fop.level == OZ_S4) filter_mv_low += mv;
        if (fop.level == OZ_S5) filter_mv_mid += mv;
        tm.mark(3);
        if ((rc = phase_qr(ctx, V, N, locked, Va, N, N, ma))) return rc;
        tm.mark(4);
        if ((rc = phase_rr(ctx, op, Va, N, ma, s.theta, B2, B3))) return rc;
        matvecs += ma;
        tm.mark(5);
        CK(launch_residuals(N, ma, B3, N, B2, N, s.theta, s.resid, (double *)ctx->part.p, ctx->sc,
                            ctx->st));
        CK(launch_chase_update(ma, nev, tol, deg_max, s.theta, s.resid, s.deg, s.perm, ctx->sc,
                               ctx->st));
        CK(launch_copy_cols(N, ma, B2, N, Va, N, s.perm, ctx->st));
        tm.mark(6);
        CK(cudaMemcpyAsync(th.data(), s.theta, ma * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(rr.data(), s.resid, ma * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(perm.data(), s.perm, ma * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(hdeg.data(), s.deg, ma * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        if ((rc = sync_scalars(ctx))) return rc;
        tm.add(1, 2, 3);
        tm.add(2, 3, 4);
        tm.add(3, 4, 5);
        tm.add(4, 5, 6);
        for (int j = 0; j < ma; j++) {
            lam[locked + j] = th[perm[j]];
            res[locked + j] = rr[perm[j]];
        }
        locked = ctx->hsc->locked;
        alpha = ctx->hsc->alpha;
        lower = ctx->hsc->lower;
        if (locked >= nev) {
            converged = true;
            break;
        }
        // nex tuner: the damping of the nev-th Ritz value (th holds the Ritz
        // values of the unlocked block in ascending order)
        if (tuner && !grown && nev - 1 - locked0 >= 0) {
            const double d = damping_of(th[nev - 1 - locked0], alpha, beta);
            if (damp_prev >= 0.0 && fabs(d - damp_prev) <= kNexSettled && d > o.nex_damping) {
                grown = true;
                const int nex2 = grown_nex(nex, nev, N);
                if (nex2 > nex) {
                    const int m2 = nev + nex2;
                    CK(launch_random_block(o.seed, 5, N, m2 - m, m, V, N, ctx->st));
                    hdeg.resize(m2, deg_max);
                    for (int j = m - locked; j < m2 - locked; j++) hdeg[j] = deg_max;
                    lam.resize(m2, alpha);
                    res.resize(m2, INFINITY);
                    th.resize(m2);
                    rr.resize(m2);
                    perm.resize(m2);
                    nex = nex2;
                    m = m2;
                }
            }
            damp_prev = d;
        }
    }
    // output: locked pairs sorted ascending
    tm.mark(2);
    std::vector<int> order(nev);
    for (int j = 0; j < nev; j++) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] < lam[b]; });
    for (int j = 0; j < nev; j++) {
        h_evals[j] = lam[order[j]];
        h_resid[j] = (order[j] < locked) ? res[order[j]] : INFINITY;
    }
    CK(cudaMemcpyAsync(s.order, order.data(), nev * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
    CK(launch_copy_cols(N, nev, V, N, d_evecs, ldz, s.order, ctx->st));
    if (op.tc) {
        // The Ritz vectors went through tensor-core products whose 48-bit
        // slices leave an orthogonality error near 1e-12; one native FP64
        // Cholesky QR pass of the nev output vectors (their Gram matrix is
        // the identity to that level) restores FP64 orthonormality.
        GenTcScope fp64(ctx, false);
        if ((rc = cholqr_pass(ctx, (z_t *)d_evecs, ldz, N, nev, 0.0))) return rc;
    }
    CK(launch_phase_normalize(N, nev, d_evecs, ldz, ctx->st));
    tm.mark(3);
    CK(cudaStreamSynchronize(ctx->st));
    harvest_kernel_times(ctx);
    tm.add(4, 2, 3);
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->iters = it;
        stats->locked = locked;
        stats->matvecs = matvecs + filter_mv;
        stats->filter_matvecs = filter_mv;
        stats->ms_lanczos = tm.acc[0];
        stats->ms_filter = tm.acc[1];
        stats->ms_qr = tm.acc[2];
        stats->ms_rr = tm.acc[3];
        stats->ms_resid = tm.acc[4];
        stats->ms_total = tm.acc[0] + tm.acc[1] + tm.acc[2] + tm.acc[3] + tm.acc[4];
        stats->filter_tflops =
            (tm.acc[1] > 0) ? 8.0 * (double)N * (double)N * (double)filter_mv / (tm.acc[1] * 1e9)
                            : 0.0;
        stats->norm_est = norm_est;
        stats->alpha = alpha;
        stats->beta = beta;
        stats->lower = lower;
        stats->kernel_launches = bse_launch_count() - launches0;
        stats->filter_launches = filter_launches;
        stats->filter_matvecs_low = filter_mv_low;
        stats->filter_matvecs_mid = filter_mv_mid;
        stats->tc_kernel_ms = ctx->k_ms;
        stats->tc_kernel_launches = ctx->k_launches;
        stats->tc_kernel_tflops = ctx->k_ms > 0 ? ctx->k_flops / (ctx->k_ms * 1e9) : 0.0;
        stats->nex_used = nex;
    }
    if (!converged) return fail(ctx, BSE_ENOCONV, "not converged after max_iter iterations%s");
    return BSE_OK;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(d);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

BseModel bse_model_of(const bse_model *model) {
    BseModel md{2.0, 0.3, 0.5, 0.01, 1.0, 8};
    if (model) {
        md.band_gap = model->band_gap;
        md.w0 = model->w0;
        md.x0 = model->x0;
        md.jitter = model->jitter;
        md.dispersion = model->dispersion;
        md.rank_x = model->rank_x;
    }
    return md;
}

namespace {

// The generator's tables in the context's workspace: u[N] and a[N R] first
// (16-byte aligned), then dE[N] and Kt[Nk/2 + 1].
int bse_tables(bsechase_ctx *ctx, uint64_t seed, int Nk, int Nv, int Nc, const BseModel &md,
               BseSource *src) {
    const int64_t N = (int64_t)Nk * Nv * Nc;
    const size_t tb = (size_t)N * (1 + std::max(md.rank_x, 1)) * sizeof(z_t) +
                      ((size_t)N + Nk / 2 + 1) * sizeof(double);
    int rc;
    if ((rc = ensure(ctx, ctx->tables, tb))) return rc;
    z_t *u = (z_t *)ctx->tables.p, *a = u + N;
    double *dE = (double *)(a + N * std::max(md.rank_x, 1)), *Kt = dE + N;
    *src = BseSource{Nk, Nv, Nc, md, dE, Kt, u, a};
    return BSE_OK;
}

}  // namespace

int bse_source(bsechase_ctx *ctx, uint64_t seed, int Nk, int Nv, int Nc, const BseModel &md,
               BseSource *src) {
    int rc;
    if ((rc = bse_tables(ctx, seed, Nk, Nv, Nc, md, src))) return rc;
    CK(launch_bse_tables(seed, Nk, Nv, Nc, md, (double *)src->dE, (z_t *)src->u, (z_t *)src->a,
                         (double *)src->Kt, ctx->st));
    return BSE_OK;
}

// =================================================================== ABI

extern "C" {

const char *bsechase_strerror(int status) {
    switch (status) {
        case BSE_OK: return "success";
        case BSE_EINVAL: return "invalid argument";
        case BSE_ENOMEM: return "out of device memory";
        case BSE_ENOCONV: return "not converged";
        case BSE_ENONFINITE: return "non-finite value or failed factorisation";
        case BSE_ETIMEOUT: return "timed out";
        case BSE_ECUDA: return "CUDA error";
        case BSE_EBUSY: return "busy";
        default: return "unknown status";
    }
}

const char *bsechase_last_error(const bsechase_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int bsechase_set_wait_limit(bsechase_ctx *ctx, double seconds) {
    if (!ctx) return BSE_EINVAL;
    if (!(seconds > 0.0) || seconds > 60.0)
        return fail(ctx, BSE_EINVAL, "wait limit must be in (0, 60] seconds%s");
    ctx->wait_ns = (uint64_t)(seconds * 1e9);
    if (ctx->wait_ns == 0) ctx->wait_ns = 1;
    return BSE_OK;
}

int bsechase_host_alloc(void **p, size_t bytes) {
    if (!p || bytes == 0) return BSE_EINVAL;
    *p = nullptr;
    if (cudaHostAlloc(p, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return BSE_ENOMEM;
    }
    return BSE_OK;
}

int bsechase_host_free(void *p) {
    if (!p) return BSE_OK;
    return cudaFreeHost(p) == cudaSuccess ? BSE_OK : BSE_ECUDA;
}

int bsechase_create(bsechase_ctx **out, int device, void *stream) {
    if (!out) return BSE_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return BSE_ECUDA;
    }
    bsechase_ctx *ctx = new (std::nothrow) bsechase_ctx();
    if (!ctx) return BSE_ENOMEM;
    ctx->device = device;
    DeviceGuard g(device);
    if (stream) {
        ctx->st = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) == cudaSuccess) {
        ctx->own_stream = true;
    } else {
        delete ctx;
        return BSE_ECUDA;
    }
    if (cudaMalloc(&ctx->sc, sizeof(ChaseScalars)) != cudaSuccess ||
        cudaMallocHost(&ctx->hsc, sizeof(ChaseScalars)) != cudaSuccess) {
        bsechase_destroy(ctx);
        return BSE_ENOMEM;
    }
    if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        ctx->sms = 152;
    ctx->ev_ok = true;
    for (int i = 0; i < kCtxEvents; i++)
        if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) ctx->ev_ok = false;
    *out = ctx;
    return BSE_OK;
}

void bsechase_destroy(bsechase_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    bse_server_shutdown(ctx);
    if (ctx->st) {
        release_workspace(ctx);
        cudaStreamSynchronize(ctx->st);
    }
    if (ctx->sc) cudaFree(ctx->sc);
    if (ctx->hsc) cudaFreeHost(ctx->hsc);
    for (int i = 0; i < kCtxEvents; i++)
        if (ctx->ev_ok) cudaEventDestroy(ctx->ev[i]);
    for (cudaEvent_t e : ctx->kev) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->st);
    delete ctx;
}

int64_t bse_dim(int Nk, int Nv, int Nc) {
    if (Nk < 1 || Nv < 1 || Nc < 1) return -1;
    const int64_t N = (int64_t)Nk * Nv * Nc;
    return N > (int64_t)1 << 31 ? -1 : N;
}

int bse_build_hamiltonian(bsechase_ctx *ctx, uint64_t seed, int Nk, int Nv, int Nc,
                          const bse_model *model, void *d_H, int64_t ldh) {
    if (!ctx) return BSE_EINVAL;
    const int64_t N = bse_dim(Nk, Nv, Nc);
    if (N < 1 || !d_H || ldh < N) return fail(ctx, BSE_EINVAL, "bad sizes or NULL H%s");
    const BseModel md = bse_model_of(model);
    if (md.rank_x < 0 || md.rank_x > 64) return fail(ctx, BSE_EINVAL, "rank_x outside 0..64%s");
    DeviceGuard g(ctx->device);
    int rc;
    BseSource t;
    if ((rc = bse_tables(ctx, seed, Nk, Nv, Nc, md, &t))) return rc;
    CK(launch_bse_build(seed, Nk, Nv, Nc, md, (double *)t.dE, (z_t *)t.u, (z_t *)t.a,
                        (double *)t.Kt, (z_t *)d_H, ldh, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return BSE_OK;
}

int chase_solve_bse(bsechase_ctx *ctx, uint64_t seed, int Nk, int Nv, int Nc,
                    const bse_model *model, int nev, int nex, double tol, int deg_max,
                    int precision, const chase_opts *opts, double *h_evals, void *d_evecs,
                    int64_t ldz, double *h_resid, chase_stats *stats) {
    if (!ctx) return BSE_EINVAL;
    const int64_t N = bse_dim(Nk, Nv, Nc);
    if (N < 1) return fail(ctx, BSE_EINVAL, "bad sizes%s");
    const BseModel md = bse_model_of(model);
    if (md.rank_x < 0 || md.rank_x > 64) return fail(ctx, BSE_EINVAL, "rank_x outside 0..64%s");
    if (!h_evals || !d_evecs || !h_resid) return fail(ctx, BSE_EINVAL, "NULL output%s");
    // the checks of chase_solve, with the (absent) matrix's place taken by an output
    int rc = validate_solve(ctx, h_evals, N, N, nev, nex, tol, deg_max, precision, ldz);
    if (rc) return rc;
    if (!precision_uses_tc(precision_mode(precision)))
        return fail(ctx, BSE_EINVAL, "the stored-H-free solve needs a tensor-core precision%s");
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    BseSource src;
    if ((rc = bse_source(ctx, seed, Nk, Nv, Nc, md, &src))) return rc;
    return solve_device(ctx, nullptr, N, N, nev, nex, tol, deg_max, precision_mode(precision),
                        opts, h_evals, (z_t *)d_evecs, ldz, h_resid, stats, &src);
}

int chase_solve(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, int nev, int nex,
                double tol, int deg_max, int precision, const chase_opts *opts, double *h_evals,
                void *d_evecs, int64_t ldz, double *h_resid, chase_stats *stats) {
    int rc = validate_solve(ctx, d_H, N, ldh, nev, nex, tol, deg_max, precision, ldz);
    if (rc) return rc;
    if (!h_evals || !d_evecs || !h_resid) return fail(ctx, BSE_EINVAL, "NULL output%s");
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    return solve_device(ctx, (const z_t *)d_H, N, ldh, nev, nex, tol, deg_max,
                        precision_mode(precision), opts,
                        h_evals, (z_t *)d_evecs, ldz, h_resid, stats);
}

int chase_solve_host(bsechase_ctx *ctx, const void *h_H, int64_t N, int64_t ldh, int nev,
                     int nex, double tol, int deg_max, int precision, const chase_opts *opts,
                     double *h_evals, void *h_evecs, int64_t ldz, double *h_resid,
                     chase_stats *stats) {
    int rc = validate_solve(ctx, h_H, N, ldh, nev, nex, tol, deg_max, precision, ldz);
    if (rc) return rc;
    if (!h_evals || !h_evecs || !h_resid) return fail(ctx, BSE_EINVAL, "NULL output%s");
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    if ((rc = ensure(ctx, ctx->Hdev, (size_t)N * N * sizeof(z_t)))) return rc;
    if ((rc = ensure(ctx, ctx->Zdev, (size_t)N * nev * sizeof(z_t)))) return rc;
    // Only the lower triangle crosses the host link (half the bytes of H; the
    // link, not HBM, bounds this copy): rows j0.. of each block of columns
    // j0.., then the upper triangle is mirrored on the device.
    z_t *Hd = (z_t *)ctx->Hdev.p;
    const z_t *Hh = (const z_t *)h_H;
    int64_t h2d = 0;
    if (ctx->ev_ok) cudaEventRecord(ctx->ev[8], ctx->st);
    for (int64_t j0 = 0; j0 < N; j0 += kHostCopyCols) {
        const int64_t w = std::min<int64_t>(kHostCopyCols, N - j0);
        CK(cudaMemcpy2DAsync(Hd + j0 + j0 * N, N * sizeof(z_t), Hh + j0 + j0 * ldh,
                             ldh * sizeof(z_t), (N - j0) * sizeof(z_t), w,
                             cudaMemcpyHostToDevice, ctx->st));
        h2d += (N - j0) * w * (int64_t)sizeof(z_t);
    }
    // half storage reads the lower triangle alone: no mirror needed
    if (!(opts && opts->half_storage == 1)) CK(launch_mirror_lower(N, Hd, N, ctx->st));
    if (ctx->ev_ok) cudaEventRecord(ctx->ev[9], ctx->st);
    rc = solve_device(ctx, (const z_t *)ctx->Hdev.p, N, N, nev, nex, tol, deg_max,
                      precision_mode(precision), opts,
                      h_evals, (z_t *)ctx->Zdev.p, N, h_resid, stats);
    if (rc != BSE_OK && rc != BSE_ENOCONV) return rc;
    CK(cudaMemcpy2DAsync(h_evecs, ldz * sizeof(z_t), ctx->Zdev.p, N * sizeof(z_t), N * sizeof(z_t),
                         nev, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (stats) {
        stats->h2d_bytes = h2d;
        stats->d2h_bytes = N * nev * (int64_t)sizeof(z_t);
        float ms = 0.f;
        if (ctx->ev_ok && cudaEventElapsedTime(&ms, ctx->ev[8], ctx->ev[9]) == cudaSuccess)
            stats->ms_h2d = ms;
    }
    return rc;
}

int chase_lanczos(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, int m, int steps,
                  int runs, uint64_t seed, int precision, double *out) {
    if (!ctx) return BSE_EINVAL;
    if (!d_H || !out || N < 1 || ldh < N || m < 1 || m > N ||
        !precision_valid(precision))
        return fail(ctx, BSE_EINVAL, "bad Lanczos arguments%s");
    DeviceGuard g(ctx->device);
    int rc;
    if ((rc = ensure_workspace(ctx, N, std::min<int64_t>(m, kMaxM)))) return rc;
    CK(cudaMemsetAsync(ctx->sc, 0, sizeof(ChaseScalars), ctx->st));
    precision = precision_mode(precision);
    Hop op{(const z_t *)d_H, N, ldh, precision_uses_tc(precision),
           precision == CHASE_MIXED_FP32 ? OZ_S4 : OZ_S6};
    if ((rc = hop_prepare(ctx, op, 8))) return rc;
    if ((rc = phase_lanczos(ctx, op, m, steps, runs, seed))) return rc;
    if ((rc = sync_scalars(ctx))) return rc;
    out[0] = ctx->hsc->beta;
    out[1] = ctx->hsc->mu_1;
    out[2] = ctx->hsc->mu_m;
    out[3] = ctx->hsc->norm_est;
    return BSE_OK;
}

int chase_filter(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, void *d_V,
                 int64_t ldv, int m, const int *h_deg, double lower, double c, double e,
                 int precision, int64_t *matvecs) {
    if (!ctx) return BSE_EINVAL;
    if (!d_H || !d_V || !h_deg || N < 1 || ldh < N || ldv != N || m < 1 || m > kMaxM || !(e > 0) ||
        !precision_valid(precision))
        return fail(ctx, BSE_EINVAL, "bad filter arguments (ldv must equal N)%s");
    for (int j = 0; j < m; j++)
        if (h_deg[j] < 1 || (j > 0 && h_deg[j] < h_deg[j - 1]))
            return fail(ctx, BSE_EINVAL, "degrees must be >= 1 and ascending%s");
    DeviceGuard g(ctx->device);
    int rc;
    if ((rc = ensure_workspace(ctx, N, m))) return rc;
    Small s = small_layout(ctx, m);
    CK(cudaMemcpyAsync(s.deg, h_deg, m * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemsetAsync(ctx->sc, 0, sizeof(ChaseScalars), ctx->st));
    precision = precision_mode(precision);
    Hop op{(const z_t *)d_H, N, ldh, precision_uses_tc(precision),
           precision == CHASE_MIXED_FP32 ? OZ_S4 : OZ_S6};
    if ((rc = hop_prepare(ctx, op, m))) return rc;
    if ((rc = phase_filter(ctx, op, (z_t *)d_V, ldv, m, h_deg, s.deg, lower, c, e, matvecs)))
        return rc;
    return sync_scalars(ctx);
}

int chase_qr(bsechase_ctx *ctx, const void *d_L, int64_t ldl, int k, void *d_V, int64_t ldv,
             int64_t N, int m) {
    if (!ctx) return BSE_EINVAL;
    if (!d_V || N < 1 || ldv < N || m < 1 || k < 0 || k + m > kMaxM || (k > 0 && (!d_L || ldl < N)))
        return fail(ctx, BSE_EINVAL, "bad QR arguments%s");
    DeviceGuard g(ctx->device);
    int rc;
    if ((rc = ensure_workspace(ctx, N, k + m))) return rc;
    CK(cudaMemsetAsync(ctx->sc, 0, sizeof(ChaseScalars), ctx->st));
    if ((rc = phase_qr(ctx, (const z_t *)d_L, ldl, k, (z_t *)d_V, ldv, N, m))) return rc;
    return sync_scalars(ctx);
}

int chase_rayleigh_ritz(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh,
                        const void *d_Q, int64_t ldq, int m, int precision, double *h_theta,
                        void *d_V, void *d_HV, double norm, double *h_resid) {
    if (!ctx) return BSE_EINVAL;
    if (!d_H || !d_Q || !h_theta || !d_V || !d_HV || N < 1 || ldh < N || ldq < N || m < 1 ||
        m > kMaxM || !precision_valid(precision))
        return fail(ctx, BSE_EINVAL, "bad Rayleigh-Ritz arguments%s");
    DeviceGuard g(ctx->device);
    int rc;
    if ((rc = ensure_workspace(ctx, N, m))) return rc;
    Small s = small_layout(ctx, m);
    CK(cudaMemsetAsync(ctx->sc, 0, sizeof(ChaseScalars), ctx->st));
    precision = precision_mode(precision);
    Hop op{(const z_t *)d_H, N, ldh, precision_uses_tc(precision),
           precision == CHASE_MIXED_FP32 ? OZ_S4 : OZ_S6};
    if ((rc = hop_prepare(ctx, op, m))) return rc;
    GenTcScope gen_scope(ctx, op.tc);
    if ((rc = phase_rr(ctx, op, (const z_t *)d_Q, ldq, m, s.theta, (z_t *)d_V, (z_t *)d_HV)))
        return rc;
    if (h_resid) {
        ChaseScalars one{};
        one.norm_est = norm;
        CK(cudaMemcpyAsync(&ctx->sc->norm_est, &one.norm_est, sizeof(double),
                           cudaMemcpyHostToDevice, ctx->st));
        CK(launch_residuals(N, m, (const z_t *)d_HV, N, (const z_t *)d_V, N, s.theta, s.resid,
                            (double *)ctx->part.p, ctx->sc, ctx->st));
        CK(cudaMemcpyAsync(h_resid, s.resid, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    }
    CK(cudaMemcpyAsync(h_theta, s.theta, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    return sync_scalars(ctx);
}

int chase_gram(bsechase_ctx *ctx, const void *d_A, int64_t lda, const void *d_B, int64_t ldb,
               int64_t K, int m1, int m2, void *d_G, int64_t ldg) {
    if (!ctx) return BSE_EINVAL;
    if (!d_A || !d_B || !d_G || K < 1 || lda < K || ldb < K || m1 < 1 || m2 < 1 || m1 > kMaxM ||
        m2 > kMaxM || ldg < m1)
        return fail(ctx, BSE_EINVAL, "bad Gram arguments%s");
    DeviceGuard g(ctx->device);
    int rc;
    if ((rc = ensure(ctx, ctx->part, (size_t)kCnWork * sizeof(z_t)))) return rc;
    CK(launch_zgemm_cn(m1, m2, K, (const z_t *)d_A, lda, (const z_t *)d_B, ldb, (z_t *)d_G, ldg,
                       0.0, 0, (z_t *)ctx->part.p, kCnWork, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return BSE_OK;
}

}  // extern "C"

namespace {

int hemm(bsechase_ctx *ctx, const Hop &hop, int n, const void *d_Y, int64_t ldy, void *d_C,
         int64_t ldc) {
    DeviceGuard g(ctx->device);
    int rc;
    CK(cudaMemsetAsync(ctx->sc, 0, sizeof(ChaseScalars), ctx->st));
    Hop op = hop;
    if ((rc = hop_prepare(ctx, op, n))) return rc;
    GemmEpi plain{};
    if ((rc = hop_apply(ctx, op, n, (const z_t *)d_Y, ldy, (z_t *)d_C, ldc, plain))) return rc;
    return sync_scalars(ctx);
}

bool hemm_args_ok(const void *d_H, int64_t N, int64_t ldh, const void *d_Y, int64_t ldy, int n,
                  const void *d_C, int64_t ldc) {
    return d_H && d_Y && d_C && N >= 1 && ldh >= N && ldy >= N && ldc >= N && n >= 1 && n <= kMaxM;
}

}  // namespace

extern "C" {

int chase_hemm(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh, const void *d_Y,
               int64_t ldy, int n, void *d_C, int64_t ldc, int precision) {
    if (!ctx) return BSE_EINVAL;
    if (!hemm_args_ok(d_H, N, ldh, d_Y, ldy, n, d_C, ldc) || !precision_valid(precision))
        return fail(ctx, BSE_EINVAL, "bad product arguments%s");
    precision = precision_mode(precision);
    const Hop op{(const z_t *)d_H, N, ldh, precision_uses_tc(precision),
                 precision == CHASE_MIXED_FP32 ? OZ_S4 : OZ_S6};
    return hemm(ctx, op, n, d_Y, ldy, d_C, ldc);
}

int chase_hemm_slices(bsechase_ctx *ctx, const void *d_H, int64_t N, int64_t ldh,
                      const void *d_Y, int64_t ldy, int n, void *d_C, int64_t ldc, int slices,
                      int half_storage) {
    if (!ctx) return BSE_EINVAL;
    if (!hemm_args_ok(d_H, N, ldh, d_Y, ldy, n, d_C, ldc) || slices < 4 || slices > 6 ||
        (half_storage != 0 && half_storage != 1))
        return fail(ctx, BSE_EINVAL, "bad product arguments%s");
    Hop op{(const z_t *)d_H, N, ldh, true, slices == 4 ? OZ_S4 : slices == 5 ? OZ_S5 : OZ_S6};
    op.tri = half_storage == 1;
    return hemm(ctx, op, n, d_Y, ldy, d_C, ldc);
}

}  // extern "C"

#include <atomic>
namespace {
std::atomic<int64_t> g_launches{0};
}
int64_t bse_launch_count() { return g_launches.load(std::memory_order_relaxed); }
void bse_count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
