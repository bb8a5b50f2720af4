// Stable LSD radix sort of (uint32 key, uint32 value) pairs and an fp32
// inclusive scan, both hand-written for sm_103a.
//
// Radix pass (8-bit digit, tiles of 2048 items = 256 threads x 8):
//   1. hist:    per-tile digit histogram (shared-memory atomics) -> counts[d][tile],
//               per-digit totals (global atomics).
//   2. scan:    one block per digit, exclusive scan of counts[d][*] over tiles.
//   3. scatter: each tile ranks its items stably (warp match_any + per-warp
//               digit counts, in index order), reorders them in shared memory by
//               digit and writes each digit's run contiguously.
// Keys are ranked by min(key, clamp), so out-of-range keys sort last.
#include <cuda_runtime.h>

#include "rll_device.cuh"
#include "rll_internal.h"

namespace rll {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;
static_assert(kTile == kSortTile, "tile size");

template <int DB>
__device__ __forceinline__ uint32_t digit_of(uint32_t key, uint32_t clamp, int shift)
{
    return (min(key, clamp) >> shift) & ((1u << DB) - 1u);
}

template <int DB>
__global__ void __launch_bounds__(kThreads) k_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                   uint32_t clamp, uint32_t* __restrict__ counts,
                                                   uint32_t* __restrict__ totals, int64_t tiles)
{
    constexpr int kDigits = 1 << DB;
    __shared__ uint32_t h[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t i = base + j * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[digit_of<DB>(keys[i], clamp, shift)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += kThreads) {
        counts[(int64_t)d * tiles + blockIdx.x] = h[d];
        if (h[d]) atomicAdd(&totals[d], h[d]);
    }
}

// exclusive scan of v over a 1024-thread block; returns the block total in *total
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t* s_warp, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0u;
    *total = s_warp[31];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t* __restrict__ counts, int64_t tiles)
{
    __shared__ uint32_t s_warp[32];
    uint32_t* row = counts + (int64_t)blockIdx.x * tiles;
    uint32_t carry = 0;
    for (int64_t b = 0; b < tiles; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < tiles ? row[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan_1024(v, s_warp, &tot);
        if (i < tiles) row[i] = carry + ex;
        carry += tot;
    }
}

// exclusive scan over kThreads * DPT values held DPT per thread (thread t
// owns entries t*DPT .. t*DPT+DPT-1); s_scan: kWarps words of scratch
template <int DPT>
__device__ __forceinline__ void block_excl_scan_owned(const uint32_t* in, uint32_t* out, uint32_t* s_scan)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t v[DPT], sum = 0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        v[k] = in[t * DPT + k];
        sum += v[k];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();  // s_scan may still be read by an earlier scan
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_scan[w];
    uint32_t run = before + x - sum;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        out[t * DPT + k] = run;
        run += v[k];
    }
}

// Stable scatter of one tile. Warp w ranks items w*256 .. w*256+255 of the
// tile (8 rounds of 32 consecutive items) with private per-digit counters
// (match_any groups equal digits; the group's first lane advances the
// counter), so no block barrier is needed per round. Then per digit the
// warps' counts are prefix-summed, items are reordered by digit in shared
// memory, and every digit's run is written contiguously.
template <int DB>
__global__ void __launch_bounds__(kThreads) k_scatter(const uint32_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      uint32_t* __restrict__ kout,
                                                      uint32_t* __restrict__ vout, int64_t n, int shift,
                                                      uint32_t clamp, const uint32_t* __restrict__ counts,
                                                      const uint32_t* __restrict__ totals, int64_t tiles)
{
    constexpr int kDigits = 1 << DB;
    constexpr int DPT = kDigits / kThreads;
    constexpr int kPerWarp = kTile / kWarps;  // 256 consecutive items per warp
    __shared__ uint32_t s_wc[kWarps][kDigits];  // per-warp counts, then per-warp offsets
    __shared__ uint32_t s_cnt[kDigits];
    __shared__ uint32_t s_start[kDigits];
    __shared__ uint32_t s_base[kDigits];
    __shared__ uint32_t s_k[kTile];
    __shared__ uint32_t s_v[kTile];
    __shared__ uint32_t s_scan[kWarps];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int w = 0; w < kWarps; ++w)
        for (int q = t; q < kDigits; q += kThreads) s_wc[w][q] = 0;
    for (int q = t; q < kDigits; q += kThreads) s_base[q] = totals[q];
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    uint32_t k[kItems], v[kItems], d[kItems], r[kItems];
    uint32_t* wc = s_wc[warp];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t i = base + warp * kPerWarp + j * 32 + lane;
        if (i < n) {
            k[j] = kin[i];
            v[j] = vin[i];
            d[j] = digit_of<DB>(k[j], clamp, shift);
        } else {
            k[j] = 0xFFFFFFFFu;
            v[j] = 0u;
            d[j] = kDigits - 1;  // padding ranks after every real item of the tile
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d[j]);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader) {
            old = wc[d[j]];
            wc[d[j]] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        r[j] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps; tile count
    for (int q = t; q < kDigits; q += kThreads) {
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = s_wc[w][q];
            s_wc[w][q] = run;
            run += c;
        }
        s_cnt[q] = run;
    }
    __syncthreads();
    block_excl_scan_owned<DPT>(s_cnt, s_start, s_scan);  // tile-local digit starts
    block_excl_scan_owned<DPT>(s_base, s_base, s_scan);  // global digit starts
    __syncthreads();
    for (int q = t; q < kDigits; q += kThreads) s_base[q] += counts[(int64_t)q * tiles + blockIdx.x];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t pos = s_start[d[j]] + s_wc[warp][d[j]] + r[j];
        s_k[pos] = k[j];
        s_v[pos] = v[j];
    }
    __syncthreads();
    const int64_t valid = min((int64_t)kTile, n - base);
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int idx = j * kThreads + t;
        if (idx < valid) {
            const uint32_t key = s_k[idx];
            const uint32_t dg = digit_of<DB>(key, clamp, shift);
            const uint32_t dst = s_base[dg] + (uint32_t)idx - s_start[dg];
            kout[dst] = key;
            vout[dst] = s_v[idx];
        }
    }
}

// ---------------------------------------------------------------- float scan
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ float block_incl_scan_f32(float v, float* s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        float w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const float before = warp > 0 ? s_warp[warp - 1] : 0.0f;
    __syncthreads();
    return before + x;
}

// each block scans kScanBlock consecutive items (kScanItems per thread,
// thread-contiguous); block totals to sums[blockIdx]
// in and out may be the same array (the block-sums pass scans in place)
__global__ void __launch_bounds__(kScanThreads) k_scan_f32(const float* in, float* out, int64_t n,
                                                           float* __restrict__ sums)
{
    __shared__ float s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    float v[kScanItems];
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? in[base + j] : 0.0f;
        acc += v[j];
        v[j] = acc;
    }
    const float incl = block_incl_scan_f32(acc, s_warp);
    const float before = incl - acc;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) out[base + j] = before + v[j];
    if (sums && threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(float* __restrict__ out, int64_t n,
                                                           const float* __restrict__ sums)
{
    if (blockIdx.x == 0) return;
    const float add = sums[blockIdx.x - 1];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) out[base + j] += add;
}

}  // namespace

size_t radix_sort_scratch_bytes(int64_t n) { return sort_scratch_bytes_for(n); }

namespace {

template <int DB>
cudaError_t sort_passes(cudaStream_t s, const uint32_t* kin, const uint32_t* vin, int64_t n, int bits, uint32_t clamp,
                        uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, uint32_t* counts, uint32_t* totals,
                        uint32_t** kout, uint32_t** vout)
{
    constexpr int kDigits = 1 << DB;
    const int64_t tiles = (n + kTile - 1) / kTile;
    const uint32_t* ck = kin;
    const uint32_t* cv = vin;
    uint32_t* dk = ka;
    uint32_t* dv = va;
    const int passes = bits <= 0 ? 1 : (bits + DB - 1) / DB;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = DB * pass;
        cudaError_t e = cudaMemsetAsync(totals, 0, sizeof(uint32_t) * kDigits, s);
        if (e != cudaSuccess) return e;
        k_hist<DB><<<(unsigned)tiles, kThreads, 0, s>>>(ck, n, shift, clamp, counts, totals, tiles);
        k_scan_tiles<<<kDigits, 1024, 0, s>>>(counts, tiles);
        k_scatter<DB><<<(unsigned)tiles, kThreads, 0, s>>>(ck, cv, dk, dv, n, shift, clamp, counts, totals, tiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ck = dk;
        cv = dv;
        dk = (dk == ka) ? kb : ka;
        dv = (dv == va) ? vb : va;
    }
    *kout = const_cast<uint32_t*>(ck);
    *vout = const_cast<uint32_t*>(cv);
    return cudaSuccess;
}

}  // namespace

cudaError_t radix_sort_pairs(cudaStream_t s, const uint32_t* kin, const uint32_t* vin, int64_t n, int bits,
                             uint32_t clamp, void* scratch, uint32_t** kout, uint32_t** vout)
{
    const int64_t tiles = (n + kTile - 1) / kTile;
    char* p = (char*)scratch;
    const size_t nb = sort_align256(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t* ka = (uint32_t*)p; p += nb;
    uint32_t* va = (uint32_t*)p; p += nb;
    uint32_t* kb = (uint32_t*)p; p += nb;
    uint32_t* vb = (uint32_t*)p; p += nb;
    uint32_t* counts = (uint32_t*)p;
    p += sort_align256(sizeof(uint32_t) * kSortMaxDigits * (size_t)(tiles > 0 ? tiles : 1));
    uint32_t* totals = (uint32_t*)p;
    if (n <= 0) {
        *kout = ka;
        *vout = va;
        return cudaSuccess;
    }
    // 9-bit digits when they save a pass (26-bit keys: 3 passes instead of 4)
    const int p8 = bits <= 0 ? 1 : (bits + 7) / 8, p9 = bits <= 0 ? 1 : (bits + 8) / 9;
    if (p9 < p8) return sort_passes<9>(s, kin, vin, n, bits, clamp, ka, va, kb, vb, counts, totals, kout, vout);
    return sort_passes<8>(s, kin, vin, n, bits, clamp, ka, va, kb, vb, counts, totals, kout, vout);
}

cudaError_t inclusive_scan_f32(cudaStream_t s, const float* in, float* out, int64_t n, void* scratch)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + kScanBlock - 1) / kScanBlock;
    if (blocks > kScanBlock) return cudaErrorInvalidValue;
    float* sums = (float*)scratch;
    k_scan_f32<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, blocks > 1 ? sums : nullptr);
    if (blocks > 1) {
        k_scan_f32<<<1, kScanThreads, 0, s>>>(sums, sums, blocks, nullptr);
        k_scan_add<<<(unsigned)blocks, kScanThreads, 0, s>>>(out, n, sums);
    }
    return cudaGetLastError();
}

}  // namespace rll
