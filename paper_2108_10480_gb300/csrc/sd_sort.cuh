// Stable LSD radix sort (8-bit digits) of key/value pairs in device memory,
// one launch per digit pass ("onesweep"): the digits of every pass are
// counted at once first (by a counting kernel, or by the kernel that makes
// the keys); each pass kernel then takes tiles in launch order from an
// atomic counter, loads its keys and values, ranks them inside the tile
// (equal digits in order, by warp match masks), publishes the tile's digit
// counts, finds the counts of all earlier tiles by a decoupled look-back
// over their published (count, flag) words, up to eight tiles a round, and
// scatters its keys stably. Each pass is launched as the programmatic
// dependent of the kernel before it. Used for the Morton order of
// primitives (64-bit keys) and of queries (32-bit keys).
//
// The look-back only waits on tiles with smaller indices, which were taken
// by blocks that already run; every wait is bounded all the same. A tile
// whose wait runs out counts its digit prefix directly instead (every key of
// the earlier tiles, read from the pass's input): slower, but the same exact
// prefix, so the sort's result never depends on the wait.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace sdsort {

constexpr int THREADS = 256;
constexpr int ITEMS = 4;
constexpr int TILE = THREADS * ITEMS;
constexpr int WARPS = THREADS / 32;
constexpr int MAX_PASSES = 8;
constexpr uint32_t FLAG_AGG = 1u << 30;     // the tile's own counts
constexpr uint32_t FLAG_PRE = 2u << 30;     // counts of tiles 0..i inclusive
constexpr uint32_t VALUE = FLAG_AGG - 1u;
// polls of an unpublished look-back word before the direct count is taken;
// a negative limit never waits (every tile but the first counts directly)
#ifndef SD_SORT_SPIN_LIMIT
#define SD_SORT_SPIN_LIMIT (1 << 21)
#endif
constexpr int SPIN_LIMIT = SD_SORT_SPIN_LIMIT;

// scratch words for sorting n keys in `passes` passes: per pass the
// (tile, digit) look-back words and 256 digit totals, then one tile counter
// per pass and an error word
constexpr size_t hist_words(size_t n, int passes = MAX_PASSES)
{
    return (size_t)passes * 256 * ((n + TILE - 1) / TILE) + (size_t)passes * 256 + 64;
}

// Programmatic dependent launch: a pass kernel is launched while the kernel
// before it on the stream still runs; each of its threads first waits until
// that kernel has completed and its writes are visible, then lets the next
// pass launch in turn. (Both are no-ops for a kernel launched without the
// attribute.) The kernel that writes the keys only lets the first pass
// launch early.
__device__ __forceinline__ void pdl_wait_and_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// where the digit totals of every pass sit in the scratch words
inline uint32_t* digit_totals(uint32_t* scratch, size_t n, int passes)
{
    return scratch + (size_t)passes * 256 * ((n + TILE - 1) / TILE);
}

// a key's digits of every pass into a block's shared histogram
template <typename K>
__device__ __forceinline__ void count_key(uint32_t (*h)[256], K k, int passes)
{
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
}

// digit totals of every pass
template <typename K>
__global__ void __launch_bounds__(THREADS) count_kernel(const K* __restrict__ keys, int n, int passes,
                                                        uint32_t* __restrict__ totals)
{
    __shared__ uint32_t h[MAX_PASSES][256];
    pdl_release();
    for (int p = 0; p < passes; ++p) h[p][threadIdx.x] = 0;
    __syncthreads();
    for (int i = blockIdx.x * THREADS + threadIdx.x; i < n; i += gridDim.x * THREADS) {
        count_key(h, keys[i], passes);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        uint32_t c = h[p][threadIdx.x];
        if (c) atomicAdd(&totals[256 * p + threadIdx.x], c);
    }
}

__device__ __forceinline__ uint32_t load_volatile(const uint32_t* p) { return *(const volatile uint32_t*)p; }



template <typename K, typename V>
__global__ void __launch_bounds__(THREADS) pass_kernel(const K* __restrict__ kin, const V* __restrict__ vin,
                                                       K* __restrict__ kout, V* __restrict__ vout, int n, int shift,
                                                       const uint32_t* __restrict__ totals, uint32_t* look,
                                                       int* tile_counter)
{
    __shared__ int s_tile;
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wsum[WARPS];
    __shared__ uint32_t run[256];
    __shared__ uint32_t cnt[WARPS][256];
    pdl_wait_and_release();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1);
    run[tid] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int base = tile * TILE;
    // every global input this tile needs, loaded at once: its keys and
    // values and the pass's digit total of digit tid
    K key[ITEMS];
    V val[ITEMS];
    unsigned dig[ITEMS];
    const uint32_t total = totals[tid];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        int i = base + r * THREADS + tid;
        bool valid = i < n;
        key[r] = valid ? kin[i] : K(0);
        val[r] = valid ? vin[i] : V(0);
    }
    // Ranks inside the tile first (rounds of THREADS keys in order, ranked by
    // warp and lane with match masks): rank[r] is the number of the tile's
    // keys with the same digit before key r, and run[d] ends as the tile's
    // count of digit d.
    const unsigned lt = (1u << lane) - 1u;
    uint32_t rank[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const bool valid = base + r * THREADS + tid < n;
        dig[r] = valid ? ((unsigned)(key[r] >> shift) & 255u) : 256u + (unsigned)lane;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) cnt[w][tid] = 0;
        __syncthreads();
        const unsigned d = dig[r];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt) == 0u) cnt[warp][d] = __popc(peers);
        __syncthreads();
        rank[r] = 0;
        if (valid) {
            uint32_t pre = run[d];
            for (int w = 0; w < warp; ++w) pre += cnt[w][d];
            rank[r] = pre + __popc(peers & lt);
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) tot += cnt[w][tid];
        run[tid] += tot;
    }
    __syncthreads();
    // publish this tile's counts, then look back for the earlier tiles',
    // up to LOOK of them per round
    const uint32_t local = run[tid];
    uint32_t* mine = look + (size_t)tile * 256 + tid;
    atomicExch(mine, (tile == 0 ? FLAG_PRE : FLAG_AGG) | local);
    uint32_t excl = 0;
    bool lost = false;
    if (tile > 0) {
        constexpr int LOOK = 8;
        int j = tile - 1;
        int spins = 0;
        lost = SPIN_LIMIT < 0;
        while (!lost) {
            uint32_t w[LOOK];
#pragma unroll
            for (int q = 0; q < LOOK; ++q)
                w[q] = j - q >= 0 ? load_volatile(look + (size_t)(j - q) * 256 + tid) : FLAG_PRE;
            int q = 0;
            bool done = false;
#pragma unroll
            for (int u = 0; u < LOOK; ++u) {
                if (done || u != q) continue;
                const uint32_t f = w[u] & ~VALUE;
                if (f == 0u) continue;          // not published yet: poll it again
                excl += w[u] & VALUE;
                if (f == FLAG_PRE) done = true;
                ++q;
            }
            if (done) break;
            if (q == 0 && ++spins > SPIN_LIMIT) lost = true;
            j -= q;
        }
    }
    // a wait that ran out: the prefix of digit tid over tiles 0..tile-1,
    // counted from the keys themselves (block-uniform branch)
    if (__syncthreads_or(lost)) {
        run[tid] = 0;
        __syncthreads();
        for (int i = tid; i < base; i += THREADS) atomicAdd(&run[(unsigned)(kin[i] >> shift) & 255u], 1u);
        __syncthreads();
        excl = run[tid];
    }
    if (tile > 0) atomicExch(mine, FLAG_PRE | (excl + local));
    // digit base: exclusive scan of the pass's digit totals
    {
        const uint32_t t = total;
        uint32_t x = t;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
        s_base[tid] = wpre + x - t + excl;
    }
    __syncthreads();
    // stable scatter
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        if (base + r * THREADS + tid < n) {
            const uint32_t dst = s_base[dig[r]] + rank[r];
            kout[dst] = key[r];
            vout[dst] = val[r];
        }
    }
}

// Sorts (k0, v0) by the low `bits` bits of the key (ceil(bits / 8) passes).
// Uses (k1, v1) as the alternate buffers; returns 0 if the result ends in
// (k0, v0), 1 if in (k1, v1). scratch needs hist_words(n, passes) words.
// With `counted`, the caller has zeroed the scratch and already added every
// key's digits to digit_totals(scratch, n, passes) (the kernel that made
// the keys counted them), so the sort starts with its first pass.
// Adds the number of kernel launches to *launches.
template <typename K, typename V>
int sort_pairs(K* k0, V* v0, K* k1, V* v1, int n, int bits, uint32_t* scratch, cudaStream_t st, int* launches,
               bool counted = false)
{
    if (n <= 1) return 0;
    const int ntiles = (n + TILE - 1) / TILE;
    const int passes = (bits + 7) / 8;
    uint32_t* look = scratch;
    uint32_t* totals = look + (size_t)passes * 256 * ntiles;
    int* counters = (int*)(totals + (size_t)passes * 256);
    if (!counted) {
        cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * hist_words(n, passes), st);
        count_kernel<K><<<std::min(ntiles, 1024), THREADS, 0, st>>>(k0, n, passes, totals);
    }
    // each pass directly follows a kernel on `st` (the counting kernel, the
    // caller's key kernel when counted, or the previous pass): launched as
    // its programmatic dependent
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntiles);
    cfg.blockDim = dim3(THREADS);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const K* ki = cur ? k1 : k0;
        const V* vi = cur ? v1 : v0;
        K* ko = cur ? k0 : k1;
        V* vo = cur ? v0 : v1;
        if (cudaLaunchKernelEx(&cfg, pass_kernel<K, V>, ki, vi, ko, vo, n, 8 * p, (const uint32_t*)(totals + 256 * p),
                               look + (size_t)p * 256 * ntiles, counters + p) != cudaSuccess) {
            cudaGetLastError();     // without the attribute: an ordinary launch
            pass_kernel<K, V><<<ntiles, THREADS, 0, st>>>(ki, vi, ko, vo, n, 8 * p, totals + 256 * p,
                                                          look + (size_t)p * 256 * ntiles, counters + p);
        }
        cur ^= 1;
    }
    *launches += (counted ? 0 : 1) + passes;
    return cur;
}

}  // namespace sdsort
