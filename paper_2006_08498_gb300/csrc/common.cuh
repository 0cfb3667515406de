// Shared device helpers of the ChASE CUDA path (sm_103a).
//
// Complex numbers are double2 (x = real, y = imaginary), the memory layout
// of C99 double complex and of torch.complex128.  Every matrix is
// column-major: element (i, j) at a[i + j * ld].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#define BSE_DEV __device__ __forceinline__

// Function attributes belong to the module loaded on each device, so the
// one-time set-ups below are kept per device (index of the current device).
constexpr int kMaxDevices = 64;
inline int current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    return dev;
}

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per kernel and
// device, under std::call_once: concurrent solver threads never launch
// before it is set.
inline cudaError_t smem_attr_once(std::once_flag (&flag)[kMaxDevices], cudaError_t (&status)[kMaxDevices],
                                  const void *kernel, int bytes) {
    const int dev = current_device();
    if (dev < 0) return cudaErrorInvalidDevice;
    std::call_once(flag[dev], [&] {
        status[dev] = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    });
    return status[dev];
}


typedef double2 z_t;
typedef float2 c_t;

BSE_DEV z_t zmk(double r, double i) { return make_double2(r, i); }
BSE_DEV z_t zadd(z_t a, z_t b) { return zmk(a.x + b.x, a.y + b.y); }
BSE_DEV z_t zsub(z_t a, z_t b) { return zmk(a.x - b.x, a.y - b.y); }
BSE_DEV z_t zmul(z_t a, z_t b) { return zmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
BSE_DEV z_t zcmul(z_t a, z_t b) { return zmk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
BSE_DEV z_t zconj(z_t a) { return zmk(a.x, -a.y); }
BSE_DEV z_t zscale(z_t a, double s) { return zmk(a.x * s, a.y * s); }
BSE_DEV double zabs2(z_t a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
BSE_DEV void zfma(z_t &acc, z_t a, z_t b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
BSE_DEV void zcfma(z_t &acc, z_t a, z_t b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based
// generator: the state is set to the key, advanced by the golden gamma, and
// the 64-bit finaliser is applied.
BSE_DEV uint64_t splitmix64(uint64_t key) {
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// Uniform in [0, 1): top 53 bits of splitmix64(seed ^ (stream << 56) ^ idx).
BSE_DEV double unif(uint64_t seed, uint64_t stream, uint64_t idx) {
    return (double)(splitmix64(seed ^ (stream << 56) ^ idx) >> 11) * 0x1.0p-53;
}

BSE_DEV double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Device-side status word written by kernels instead of trapping.
enum DevError : int {
    DEV_OK = 0,
    DEV_CHOL_FAIL = 1,     // non-positive Cholesky pivot
    DEV_EIG_NOCONV = 2,    // small eigensolver did not converge
    DEV_NONFINITE = 3,     // NaN or Inf met in a reduction
    DEV_BAD_ARG = 4,       // a kernel got an argument outside its limits
    DEV_TIMEOUT = 5,       // a bounded wait inside a kernel expired
};

// Scalars shared between the kernels of one solve (device resident).
struct ChaseScalars {
    int error;         // DevError of the first failure
    int error_where;   // kernel-specific detail (column, sweep, ...)
    int locked;        // number of locked pairs
    int new_locked;    // pairs locked by the last Rayleigh-Ritz step
    int m_act;         // active (unlocked) columns
    int pad0;
    double alpha;      // lower end of the damped interval
    double beta;       // upper bound of the spectrum (Lanczos)
    double lower;      // normalisation point of the filter (min Ritz value)
    double mu_1, mu_m; // Lanczos estimates of lambda_1 and lambda_m
    double norm_est;   // ||H|| estimate used to normalise residuals
};

// Process-wide count of kernel launches issued by this library.
int64_t bse_launch_count();
void bse_count_launches(int n);

BSE_DEV void set_error(ChaseScalars *s, int code, int where) {
    if (atomicCAS(&s->error, 0, code) == 0) s->error_where = where;
}
