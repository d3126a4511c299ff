// Issue-rate probes of the pipes the pair kernel runs on (no counterpart in
// the paper): they measure the denominators of the benchmark's roofline on
// the GPU at hand.  Each thread runs 8 independent dependency chains of one
// operation (FP32 fused multiply-add, FP32 reciprocal square root on the
// special-function unit, FP64 fused multiply-add) for `iters` rounds and
// writes one value so that nothing is optimised away.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lcdm.h"

namespace {

__global__ void probe_ffma(float* out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = (float)(threadIdx.x + j);
#pragma unroll 1
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int j = 0; j < 8; j++) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_mufu(float* out, int iters) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = 1.0f + (float)(threadIdx.x + j) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int j = 0; j < 8; j++) x[j] = rsqrtf(x[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_dfma(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = (double)(threadIdx.x + j);
#pragma unroll 1
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int j = 0; j < 8; j++) x[j] = fma(x[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

int64_t lcdm_probe_ops_per_thread(int32_t iters) { return (int64_t)iters * 16 * 8; }

lcdm_status lcdm_probe(int32_t what, void* out, int32_t blocks, int32_t threads, int32_t iters,
                       cudaStream_t stream) {
    if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || (threads % 32) != 0 || iters <= 0 ||
        what < 0 || what > 2)
        return LCDM_ERR_INVALID;
    if (what == 0) probe_ffma<<<blocks, threads, 0, stream>>>((float*)out, iters, 0.999999f, 1e-7f);
    if (what == 1) probe_mufu<<<blocks, threads, 0, stream>>>((float*)out, iters);
    if (what == 2) probe_dfma<<<blocks, threads, 0, stream>>>((double*)out, iters, 0.999999999, 1e-12);
    return cudaGetLastError() == cudaSuccess ? LCDM_OK : LCDM_ERR_CUDA;
}

}  // extern "C"
