// The solver context shared by the host-side files of the library
// (chase.cu: solver and C ABI; serve.cu: request server).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/bsechase.h"
#include "kernels.h"

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct BseServer;

constexpr int kCtxEvents = 10;

struct bsechase_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    ChaseScalars *sc = nullptr;      // device
    ChaseScalars *hsc = nullptr;     // pinned host mirror
    // workspace
    DevBuf V, B1, B2, B3, G, R, Ri, Yr, heev, small_d, ints, part, lz, tables, Hdev, Zdev;
    DevBuf ozA, ozE, ozB, ozF, ozP;  // tensor-core products: slices of H and of the operand,
                                     // split-K partials
    DevBuf ozGA, ozGE;               // slices and exponents of op(A) for the general products
    DevBuf ozT;                      // half storage: the row scales t and s = 1 / t
    bool gen_tc = false;             // N x m products of QR and Rayleigh-Ritz on the tensor cores
    int sms = 0;                     // multiprocessors of the device
    uint64_t wait_ns = kDefaultWaitNs;  // bounded waits of the tensor-core kernel
    OzakiH oh;
    int64_t wsN = 0;
    int wsM = 0;
    cudaEvent_t ev[kCtxEvents];   // 0..6: solve phases; 8, 9: host copies
    bool ev_ok = false;
    // CUDA-event timing of every tensor-core product launch: event pairs
    // recorded on st, read back at the solver's synchronisation points
    std::vector<cudaEvent_t> kev;
    std::vector<double> kev_flops;   // tensor flops of each recorded launch
    size_t kev_used = 0;             // events recorded since the last harvest
    double k_ms = 0.0, k_flops = 0.0;
    int64_t k_launches = 0;
    BseServer *server = nullptr;     // request server attached to this context
    OzBatcher *batcher = nullptr;    // a server slot's shared product batcher
};

// Record a failure message (printf-style with one string argument).
int fail(bsechase_ctx *c, int code, const char *fmt, const char *detail = "");
// Grow / free the context's workspace (stream-ordered on ctx->st).
int ensure(bsechase_ctx *ctx, DevBuf &b, size_t bytes);
void release_workspace(bsechase_ctx *ctx);
// The synthetic Hamiltonian as the solve's operator without H stored: its
// parameters and the generator's tables (tensor-core precisions only).
struct BseSource {
    int Nk, Nv, Nc;
    BseModel md;
    const double *dE, *Kt;
    const z_t *u, *a;
};
// The model parameters of a bse_model (NULL: the defaults), and the
// generator's tables of (seed, Nk, Nv, Nc, md) written into the context's
// workspace as the source of a solve without the stored H.
BseModel bse_model_of(const bse_model *model);
int bse_source(bsechase_ctx *ctx, uint64_t seed, int Nk, int Nv, int Nc, const BseModel &md,
               BseSource *src);
// The whole solve on device buffers (chase_solve without argument checks);
// with `bse` set, H is that source's and `H` is unused.
int solve_device(bsechase_ctx *ctx, const z_t *H, int64_t N, int64_t ldh, int nev, int nex,
                 double tol, int deg_max, int precision, const chase_opts *opts, double *h_evals,
                 z_t *d_evecs, int64_t ldz, double *h_resid, chase_stats *stats,
                 const BseSource *bse = nullptr);
// Whether `precision` is a chase_precision value, and the mode it runs
// (CHASE_MIXED_BF16X3 runs as CHASE_MIXED_FP32).
bool precision_valid(int precision);
int precision_mode(int precision);
// Whether a (mode) precision computes the products with H on the tensor cores.
bool precision_uses_tc(int precision);
// Add the recorded tensor-core launch times to k_ms / k_flops / k_launches
// (the stream must have been synchronised) and recycle the events.
void harvest_kernel_times(bsechase_ctx *ctx);
// Stop and free the request server of a context (no-op without one).
void bse_server_shutdown(bsechase_ctx *ctx);
