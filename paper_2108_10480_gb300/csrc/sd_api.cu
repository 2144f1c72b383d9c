// Small C-ABI helpers of libsd: option defaults, status text, last error.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "sd_common.cuh"

#include <atomic>

namespace {
thread_local char g_last_error[256] = "";
std::atomic<long long> g_launches{0};
}

void sd_count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

extern "C" int64_t sd_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

void sd_set_last_error(const char* msg)
{
    std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg ? msg : "");
}

int sd_cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return SD_OK;
    sd_set_last_error(cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return SD_ERR_OOM;
    return SD_ERR_CUDA;
}

extern "C" void sd_default_build_opts(sd_build_opts* o)
{
    if (!o) return;
    o->alpha_u = 0.f;
    o->leaf_size = 1;
    o->weights = SD_WEIGHTS_PAPER;
    o->paper_metric = 0;
    o->defer_checks = 0;
}

extern "C" void sd_default_query_opts(sd_query_opts* o)
{
    if (!o) return;
    o->sort_queries = 1;
    o->block = 0;
    o->counts = nullptr;
    o->order = nullptr;
}

extern "C" const char* sd_status_str(int s)
{
    switch (s) {
    case SD_OK: return "ok";
    case SD_ERR_INVALID_ARG: return "invalid argument";
    case SD_ERR_CUDA: return "CUDA error";
    case SD_ERR_OOM: return "out of device memory";
    case SD_ERR_NONFINITE: return "non-finite coordinate";
    case SD_ERR_INDEX: return "primitive index out of range";
    case SD_ERR_TOO_LARGE: return "size too large";
    case SD_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

extern "C" const char* sd_last_error(void) { return g_last_error; }
