// Pipe-throughput probes: the denominators of the traversal's roofline.
//
// The Barnes-Hut traversal is bound by the FP32 pipe with the MUFU
// (special-function) pipe as a co-bound; neither peak is published per
// clock for this part, so they are measured here at whatever clock the GPU
// runs: every thread of a full-occupancy grid runs eight independent
// dependency chains of one instruction kind in inline PTX (so the compiler
// can neither fold nor re-associate them), and the caller times the launch
// with CUDA events.
#include <cuda_runtime.h>

#include "sd_common.cuh"

namespace {

constexpr int PB_THREADS = 256;
constexpr int PB_CHAINS = 8;
constexpr int PB_UNROLL = 16;

// a <- a * x + y on eight chains
__global__ void __launch_bounds__(PB_THREADS) k_probe_ffma(int iters, float x, float y, float* sink)
{
    float a[PB_CHAINS];
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) a[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PB_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < PB_CHAINS; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(x), "f"(y));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) s += a[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the packed two-wide form (fma.rn.f32x2): two FMAs per lane per instruction
__global__ void __launch_bounds__(PB_THREADS) k_probe_ffma2(int iters, float x, float y, float* sink)
{
    unsigned long long a[PB_CHAINS];
    unsigned long long xx, yy;
    asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(x));
    asm("mov.b64 %0, {%1, %1};" : "=l"(yy) : "f"(y));
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) {
        float lo = (float)(threadIdx.x + c), hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[c]) : "f"(lo), "f"(hi));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PB_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < PB_CHAINS; ++c)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[c]) : "l"(xx), "l"(yy));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[c]));
        s += lo + hi;
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// a <- 2^a, then a <- a * x + y (the FMA keeps the chain bounded; it issues
// on the FP32 pipe, whose rate is eight times the MUFU's, so the MUFU stays
// the bound)
__global__ void __launch_bounds__(PB_THREADS) k_probe_ex2(int iters, float x, float y, float* sink)
{
    float a[PB_CHAINS];
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) a[c] = -1.f - 0.01f * (float)c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PB_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < PB_CHAINS; ++c) {
                asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
                asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(x), "f"(y));
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) s += a[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int sd_peak_probe(int32_t kind, int32_t blocks, int32_t iters, float* sink, double* ops, void* stream)
{
    if (kind < 0 || kind > 2 || blocks <= 0 || iters <= 0 || !sink || !ops) return SD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // lane operations per launch: FMAs (kinds 0, 1) or exponentials (kind 2)
    *ops = (double)blocks * PB_THREADS * (double)iters * PB_UNROLL * PB_CHAINS * (kind == 1 ? 2.0 : 1.0);
    if (kind == 0) k_probe_ffma<<<blocks, PB_THREADS, 0, st>>>(iters, 0.999f, 1e-3f, sink);
    else if (kind == 1) k_probe_ffma2<<<blocks, PB_THREADS, 0, st>>>(iters, 0.999f, 1e-3f, sink);
    else k_probe_ex2<<<blocks, PB_THREADS, 0, st>>>(iters, -0.5f, 0.1f, sink);
    sd_count_launches(1);
    return sd_cuda_status(cudaGetLastError());
}
