// Stable LSD radix sort (8-bit digits) of key/value pairs in device memory.
// Per pass: a per-tile digit histogram (plus digit totals), an exclusive
// scan over (digit, tile) with one block per digit, and a stable scatter
// that ranks equal digits inside a tile with warp match masks. Used for the Morton order of primitives (64-bit
// keys) and of queries (32-bit keys).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdsort {

constexpr int THREADS = 256;
constexpr int ITEMS = 4;
constexpr int TILE = THREADS * ITEMS;
constexpr int WARPS = THREADS / 32;

template <typename K>
__global__ void __launch_bounds__(THREADS) hist_kernel(const K* __restrict__ keys, int n, int shift,
                                                       uint32_t* __restrict__ hist, int ntiles,
                                                       uint32_t* __restrict__ tot)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * TILE;
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        int i = base + r * THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    uint32_t c = h[threadIdx.x];
    hist[threadIdx.x * ntiles + blockIdx.x] = c;
    if (c) atomicAdd(&tot[threadIdx.x], c);
}

// Exclusive scan of the (digit, tile) counters, one block per digit: the
// digit's base is the sum of the totals of all smaller digits, and the
// block scans its row of per-tile counts (contiguous in memory).
static __global__ void __launch_bounds__(256) scan_rows_kernel(uint32_t* __restrict__ hist, int ntiles,
                                                              const uint32_t* __restrict__ tot)
{
    __shared__ uint32_t wsum[8];
    __shared__ uint32_t sbase;
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        uint32_t acc = 0;
        for (int k = lane; k < d; k += 32) acc += tot[k];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) sbase = acc;
    }
    __syncthreads();
    uint32_t carry = sbase;
    uint32_t* row = hist + (size_t)d * ntiles;
    for (int c0 = 0; c0 < ntiles; c0 += 256 * 8) {
        int b = c0 + tid * 8;
        uint32_t v[8];
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = (b + k < ntiles) ? row[b + k] : 0u;
            s += v[k];
        }
        uint32_t x = s;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t wpre = 0, total = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            uint32_t ws = wsum[w];
            if (w < warp) wpre += ws;
            total += ws;
        }
        uint32_t run = carry + wpre + x - s;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (b + k < ntiles) row[b + k] = run;
            run += v[k];
        }
        carry += total;
        __syncthreads();
    }
}

template <typename K, typename V>
__global__ void __launch_bounds__(THREADS) scatter_kernel(const K* __restrict__ kin, const V* __restrict__ vin,
                                                          K* __restrict__ kout, V* __restrict__ vout, int n,
                                                          int shift, const uint32_t* __restrict__ hist, int ntiles)
{
    __shared__ uint32_t goff[256];
    __shared__ uint32_t run[256];
    __shared__ uint32_t cnt[WARPS][256];
    int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    goff[tid] = hist[tid * ntiles + blockIdx.x];
    run[tid] = 0;
    unsigned lt = (1u << lane) - 1u;
    int base = blockIdx.x * TILE;
    for (int r = 0; r < ITEMS; ++r) {
#pragma unroll
        for (int w = 0; w < WARPS; ++w) cnt[w][tid] = 0;
        __syncthreads();
        int i = base + r * THREADS + tid;
        bool valid = i < n;
        K key = valid ? kin[i] : K(0);
        unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 256u + (unsigned)lane;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        bool leader = (peers & lt) == 0u;
        if (valid && leader) cnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = run[d];
            for (int w = 0; w < warp; ++w) pre += cnt[w][d];
            uint32_t dst = goff[d] + pre + rank;
            kout[dst] = key;
            vout[dst] = vin[i];
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) tot += cnt[w][tid];
        run[tid] += tot;
        __syncthreads();
    }
}

// counters for one sort: per-(digit, tile) counts, then 8 x 256 digit totals
inline size_t hist_words(int n) { return (size_t)256 * (size_t)((n + TILE - 1) / TILE) + 8 * 256; }

// Sorts (k0, v0) by the low `bits` bits of the key (a multiple of 8 is not
// required; passes cover ceil(bits / 8) digits). Uses (k1, v1) as the
// alternate buffers; returns 0 if the result ends in (k0, v0), 1 if in
// (k1, v1). hist needs hist_words(n) words. Adds the number of kernel
// launches to *launches.
template <typename K, typename V>
int sort_pairs(K* k0, V* v0, K* k1, V* v1, int n, int bits, uint32_t* hist, cudaStream_t st, int* launches)
{
    if (n <= 1) return 0;
    int ntiles = (n + TILE - 1) / TILE;
    int passes = (bits + 7) / 8;
    uint32_t* tot = hist + (size_t)256 * ntiles;
    cudaMemsetAsync(tot, 0, sizeof(uint32_t) * 256 * passes, st);
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        const K* ki = cur ? k1 : k0;
        const V* vi = cur ? v1 : v0;
        K* ko = cur ? k0 : k1;
        V* vo = cur ? v0 : v1;
        hist_kernel<K><<<ntiles, THREADS, 0, st>>>(ki, n, shift, hist, ntiles, tot + 256 * p);
        scan_rows_kernel<<<256, 256, 0, st>>>(hist, ntiles, tot + 256 * p);
        scatter_kernel<K, V><<<ntiles, THREADS, 0, st>>>(ki, vi, ko, vo, n, shift, hist, ntiles);
        cur ^= 1;
        *launches += 3;
    }
    return cur;
}

}  // namespace sdsort
