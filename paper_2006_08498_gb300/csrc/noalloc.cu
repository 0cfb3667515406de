// An allocation-free form of the Gram product G = A^H B.
//
// Some callers cannot allocate device memory when they call into this
// library: an application whose own memory manager has taken the device's
// memory and forbids other allocations, or a latency-bound loop that cannot
// afford cudaMalloc/cudaFree (they may synchronise the whole device), or a
// caller that cannot create a bsechase context because creating one
// allocates workspace.  chase_gram_noalloc serves them: it runs the same
// split-K kernels as chase_gram, but its partial sums live in one fixed,
// file-scope device array instead of context-owned workspace, so the call
// allocates nothing.
//
// Set-up: the first call made on a device looks up the array's device
// address (cudaGetSymbolAddress) with that device current; make that first
// call before any stream capture begins.
//
// The array holds kNoAllocScratchElems complex doubles (4 MiB) on every GPU
// that loads this library, for as long as the library stays loaded.  Every
// call shares it and it keeps the last call's contents; the kernels write
// every partial they later read, so nothing needs clearing.  Two calls whose
// work overlaps on the GPU (different streams, or different host threads on
// one device) race on the array and must be serialised by the caller.
#include <mutex>

#include "../../include/bsechase.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int64_t kNoAllocScratchElems = (int64_t)1 << 18;   // 262144 x 16 B = 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) z_t g_noalloc_scratch[kNoAllocScratchElems];

// Device address of g_noalloc_scratch, per device.  In host code the name
// g_noalloc_scratch is only a host-side handle, never a device address, so
// the address is looked up with cudaGetSymbolAddress while the device is
// current, once per device, on the first call made on that device.
std::mutex g_mu;
z_t *g_addr[kMaxDevices];

int scratch_address(int device, z_t **out) {
    if (device < 0 || device >= kMaxDevices) return BSE_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return BSE_ECUDA;
        }
        g_addr[device] = (z_t *)p;
    }
    *out = g_addr[device];
    return BSE_OK;
}

}  // namespace

extern "C" int chase_gram_noalloc(const void *d_A, int64_t lda, const void *d_B, int64_t ldb,
                                  int64_t K, int m1, int m2, void *d_G, int64_t ldg,
                                  void *cuda_stream) {
    if (!d_A || !d_B || !d_G || K < 1 || lda < K || ldb < K || m1 < 1 || m2 < 1 || ldg < m1)
        return BSE_EINVAL;
    // one split must fit: m1 * m2 partials (m1, m2 <= 512 always do)
    if (m1 > 512 || m2 > 512 || (int64_t)m1 * m2 > kNoAllocScratchElems) return BSE_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return BSE_ECUDA;
    }
    z_t *scratch = nullptr;
    int rc = scratch_address(device, &scratch);
    if (rc != BSE_OK) return rc;
    cudaError_t e = launch_zgemm_cn(m1, m2, K, (const z_t *)d_A, lda, (const z_t *)d_B, ldb,
                                    (z_t *)d_G, ldg, 0.0, 0, scratch, kNoAllocScratchElems,
                                    (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? BSE_OK : BSE_ECUDA;
}
