// Issue-rate probes for the roofline denominators of the FP64 kernels:
// DFMA and DMMA (mma.sync f64) loops, and an FFMA loop for context.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -DHAVE_M16N8K16
// Prints one JSON object per probe (TFLOP/s from CUDA events).
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
__global__ void dfma_loop(double *out, double a, double b) {
    double x[8];
    for (int i = 0; i < 8; i++) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < ITERS; it++)
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = fma(x[i], a, b);
    double s = 0; for (int i = 0; i < 8; i++) s += x[i];
    if (s == 1234.5) out[0] = s;
}
__global__ void ffma_loop(float *out, float a, float b) {
    float x[16];
    for (int i = 0; i < 16; i++) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < ITERS; it++)
#pragma unroll
        for (int i = 0; i < 16; i++) x[i] = fmaf(x[i], a, b);
    float s = 0; for (int i = 0; i < 16; i++) s += x[i];
    if (s == 1234.5f) out[0] = s;
}
__global__ void dmma884_loop(double *out) {
    double a = threadIdx.x * 1e-3, b = 1.0 - threadIdx.x * 1e-4;
    double c[4][2];
    for (int i = 0; i < 4; i++) { c[i][0] = 0; c[i][1] = 0; }
    for (int it = 0; it < ITERS; it++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
    double s = 0; for (int i = 0; i < 4; i++) s += c[i][0] + c[i][1];
    if (s == 1234.5) out[0] = s;
}
#ifdef HAVE_M16N8K16
__global__ void dmma16816_loop(double *out) {
    double a[8], b[4], c[2][4];
    for (int i = 0; i < 8; i++) a[i] = threadIdx.x * 1e-3 + i;
    for (int i = 0; i < 4; i++) b[i] = 1.0 - i * 1e-4;
    for (int i = 0; i < 2; i++) for (int j = 0; j < 4; j++) c[i][j] = 0;
    for (int it = 0; it < ITERS / 4; it++)
#pragma unroll
        for (int i = 0; i < 2; i++)
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
                         : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
                         : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                           "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
    double s = 0; for (int i = 0; i < 2; i++) for (int j = 0; j < 4; j++) s += c[i][j];
    if (s == 1234.5) out[0] = s;
}
#endif
template <class F> float timeit(F f) {
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    f(); cudaDeviceSynchronize();
    cudaEventRecord(e0); for (int r = 0; r < 3; r++) f(); cudaEventRecord(e1);
    cudaEventSynchronize(e1); float ms; cudaEventElapsedTime(&ms, e0, e1); return ms / 3;
}
int main() {
    double *d; cudaMalloc(&d, 64);
    int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * 8, threads = 256;
    float ms = timeit([&] { dfma_loop<<<blocks, threads>>>(d, 1.0000001, 1e-9); });
    double fl = 2.0 * 8 * ITERS * (double)blocks * threads;
    printf("{\"probe\":\"dfma\",\"tflops\":%.4f,\"ms\":%.3f}\n", fl / ms / 1e9, ms);
    ms = timeit([&] { ffma_loop<<<blocks, threads>>>((float *)d, 1.0000001f, 1e-9f); });
    fl = 2.0 * 16 * ITERS * (double)blocks * threads;
    printf("{\"probe\":\"ffma\",\"tflops\":%.4f,\"ms\":%.3f}\n", fl / ms / 1e9, ms);
    ms = timeit([&] { dmma884_loop<<<blocks, threads>>>(d); });
    fl = 2.0 * 8 * 8 * 4 * 4 * ITERS * (double)blocks * (threads / 32);
    printf("{\"probe\":\"dmma_m8n8k4\",\"tflops\":%.4f,\"ms\":%.3f}\n", fl / ms / 1e9, ms);
#ifdef HAVE_M16N8K16
    ms = timeit([&] { dmma16816_loop<<<blocks, threads>>>(d); });
    fl = 2.0 * 16 * 8 * 16 * 2 * (ITERS / 4) * (double)blocks * (threads / 32);
    printf("{\"probe\":\"dmma_m16n8k16\",\"tflops\":%.4f,\"ms\":%.3f}\n", fl / ms / 1e9, ms);
#endif
    cudaError_t e = cudaDeviceSynchronize();
    printf("{\"probe\":\"status\",\"err\":\"%s\",\"sms\":%d}\n", cudaGetErrorString(e), sms);
    return e != cudaSuccess;
}
