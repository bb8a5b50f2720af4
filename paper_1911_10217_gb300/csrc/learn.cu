// End-of-pass learning (Section 3, Eq. 1 and Eq. 2) and split-collapse
// (Section 3, Fig. "TreeCuts"; Section 3.1).
//
// learn_update (records bucketed by cell, then sorted per cell):
//   1. count: one thread per record; the lanes of a warp that hold the same
//      cell add their count with one atomic on the cell's cursor, and the
//      first adder of a cell appends it to the touched-cell list;
//   2. claim: every touched cell takes a contiguous bucket of its record
//      count (one atomic per warp) and its cursor becomes the bucket start;
//   3. scatter: every record writes its sample id at its cell's cursor (a
//      warp's peers take consecutive places);
//   4. one warp per touched cell orders its bucket in shared memory: a
//      counting sort by cluster, then each record's rank by sample id inside
//      its cluster group (groups are small), which gives (cluster, sample)
//      order; it then walks the records 32 at a time: a segmented inclusive
//      scan (by cluster) composes the affine maps q -> (1 - alpha) q +
//      alpha |c| of Eq. 1 in sample order, and the last lane of each segment
//      applies the composite to the cluster's Q held in shared memory; the
//      row is then stored in the table precision and its cdf rebuilt (Eq. 2
//      with the floor, prefix sum across the warp). Cells with more records
//      than a warp's buffer go to one block each: (cluster, sample id, index)
//      keys sorted by a bitonic network in shared memory (up to 8192
//      records; in place in global memory above that), then warps compose
//      different clusters in parallel.
// The order inside a bucket depends on thread scheduling; the per-cell sort
// restores sample order, so the result is deterministic.
//
// learn_update_with_scratch (the allocation-free entry point) keeps the
// earlier form: a stable radix sort of all records by key = slot * M +
// cluster, then the first record of every cell is marked (k_cell_heads) and
// one warp per cell composes the same way.
//
// split_collapse: one warp per touched cell (the paper uses one thread group
// per cell): warp arg-max over the leaves that are not single lights, warp
// arg-min over parents whose two children are both cut leaves, the
// threshold test, then one lane emits the new cut and the cdf is rebuilt.
#include <cuda_runtime.h>

#include <mutex>

#include "learn_core.cuh"
#include "rll_device.cuh"
#include "rll_internal.h"

namespace rll {
namespace {

constexpr int kWarpsPerBlock = 8;

// one warp: the default row (Q = q_init, C by Eq. 2)
template <int P>
__global__ void k_default_row(uint32_t m, float q_init, float eps, typename Store<P>::T* def_Q,
                              typename Store<P>::T* def_C)
{
    __shared__ float s_q[kMaxCut], s_c[kMaxCut];
    __shared__ uint16_t s_b[kMaxCut];
    for (uint32_t s = threadIdx.x; s < m; s += 32) {
        const typename Store<P>::T v = Store<P>::store(q_init);
        def_Q[s] = v;
        s_q[s] = Store<P>::load(v);
    }
    __syncwarp();
    warp_rebuild_cdf<P>(s_q, (int)m, eps, def_C, s_c, s_b);
}

template <int P>
__global__ void k_fill_rows(int64_t total, uint32_t M, uint32_t m, const uint32_t* __restrict__ def_cut,
                            const typename Store<P>::T* __restrict__ def_Q,
                            const typename Store<P>::T* __restrict__ def_C, uint32_t* __restrict__ cut,
                            typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = (uint32_t)(i % M);
        if (s < m) {
            cut[i] = def_cut[s];
            Q[i] = def_Q[s];
            C[i] = def_C[s];
        } else {
            cut[i] = 0u;
            Q[i] = Store<P>::store(0.0f);
            C[i] = Store<P>::store(0.0f);
        }
    }
}

// rows of empty slots hold the initial cut (a cell created later starts from it)
template <int P>
__global__ void k_reset_empty_rows(int64_t total, uint32_t M, uint32_t m, const unsigned long long* __restrict__ keys,
                                   const uint32_t* __restrict__ def_cut, const typename Store<P>::T* __restrict__ def_Q,
                                   const typename Store<P>::T* __restrict__ def_C, uint32_t* __restrict__ cut,
                                   typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = (uint32_t)(i % M);
        if (keys[i / M] != kEmptyKey) continue;
        if (s < m) {
            cut[i] = def_cut[s];
            Q[i] = def_Q[s];
            C[i] = def_C[s];
        } else {
            cut[i] = 0u;
            Q[i] = Store<P>::store(0.0f);
            C[i] = Store<P>::store(0.0f);
        }
    }
}

template <int P>
__global__ void k_to_float(int64_t total, const typename Store<P>::T* __restrict__ Q,
                           const typename Store<P>::T* __restrict__ C, float* __restrict__ q, float* __restrict__ c)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        if (q) q[i] = Store<P>::load(Q[i]);
        if (c) c[i] = Store<P>::load(C[i]);
    }
}

template <int P>
__global__ void k_from_float(int64_t total, const float* __restrict__ q, const float* __restrict__ c,
                             typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        Q[i] = Store<P>::store(q[i]);
        C[i] = Store<P>::store(c[i]);
    }
}

// one block of 256 threads covers 256 * kHeadItems sorted records; one
// global atomic per block reserves the block's share of the touched list
constexpr int kHeadItems = 8;
__global__ void __launch_bounds__(256) k_cell_heads(const uint32_t* __restrict__ sk, int64_t n, uint32_t HM, uint32_t M,
                                                    uint32_t* __restrict__ touched, uint32_t* __restrict__ touched_start,
                                                    uint32_t* __restrict__ n_touched)
{
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base_i = (int64_t)blockIdx.x * 256 * kHeadItems;
    bool head[kHeadItems];
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kHeadItems; ++j) {
        const int64_t i = base_i + (int64_t)j * 256 + threadIdx.x;
        head[j] = false;
        if (i < n) {
            const uint32_t key = sk[i];
            if (key < HM) head[j] = (i == 0) || (sk[i - 1] / M != key / M);
        }
        cnt += head[j];
    }
    // block exclusive scan of the per-thread counts
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t v = s_warp[w];
            s_warp[w] = tot;
            tot += v;
        }
        s_base = tot ? atomicAdd(n_touched, tot) : 0u;
    }
    __syncthreads();
    uint32_t slot = s_base + s_warp[warp] + x - cnt;
#pragma unroll
    for (int j = 0; j < kHeadItems; ++j) {
        if (!head[j]) continue;
        const int64_t i = base_i + (int64_t)j * 256 + threadIdx.x;
        touched[slot] = sk[i] / M;
        touched_start[slot] = (uint32_t)i;
        ++slot;
    }
}

// every occupied slot becomes a touched cell (after an import)
__global__ void k_mark_occupied(const unsigned long long* __restrict__ keys, uint32_t H, uint32_t* __restrict__ touched,
                                uint32_t* __restrict__ n_touched)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool occ = i < H && keys[i] != kEmptyKey;
    const uint32_t mask = __ballot_sync(0xffffffffu, occ);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(n_touched, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    if (occ) touched[base + __popc(mask & lanemask_lt())] = i;
}

// record key slot * M + cluster of one grid
struct GridKey {
    uint32_t HM, M, cell;
    __device__ __forceinline__ bool same(uint32_t k) const { return k < HM && k / M == cell; }
    __device__ __forceinline__ uint32_t cluster(uint32_t k) const { return k % M; }
};

template <int P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_learn_cells(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv, int64_t n, uint32_t HM,
              uint32_t M, uint32_t m, const uint32_t* __restrict__ touched,
              const uint32_t* __restrict__ touched_start, const uint32_t* __restrict__ n_touched,
              typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C, float alpha, float eps)
{
    __shared__ float s_q[kWarpsPerBlock][kMaxCut];
    __shared__ float s_c[kWarpsPerBlock][kMaxCut];
    __shared__ uint16_t s_b[kWarpsPerBlock][kMaxCut];
    const int warp = threadIdx.x >> 5;
    const uint32_t total = *n_touched;
    for (uint32_t w = blockIdx.x * kWarpsPerBlock + warp; w < total; w += gridDim.x * kWarpsPerBlock) {
        const uint32_t cell = touched[w];
        const GridKey key{HM, M, cell};
        learn_one_cell<P>(sk, sv, n, touched_start[w], key, Q + (int64_t)cell * M, C + (int64_t)cell * M, m, alpha,
                          eps, s_q[warp], s_c[warp], s_b[warp]);
    }
}

template <int P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_split(uint32_t M, uint32_t m, const uint32_t* __restrict__ touched, const uint32_t* __restrict__ n_touched,
        uint32_t* __restrict__ cut, typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C,
        const NodeRec* __restrict__ nodes, const int32_t* __restrict__ parent,
        const int32_t* __restrict__ left, const int32_t* __restrict__ right, float T, float eps,
        uint32_t max_iter, int64_t n_nodes, uint32_t* __restrict__ status)
{
    __shared__ float s_q[kWarpsPerBlock][kMaxCut];
    __shared__ float s_c[kWarpsPerBlock][kMaxCut];
    __shared__ uint32_t s_cut[kWarpsPerBlock][kMaxCut];
    __shared__ uint32_t s_nc[kWarpsPerBlock][kMaxCut];
    __shared__ uint16_t s_b[kWarpsPerBlock][kMaxCut];
    const int warp = threadIdx.x >> 5;
    const uint32_t total = *n_touched;
    for (uint32_t w = blockIdx.x * kWarpsPerBlock + warp; w < total; w += gridDim.x * kWarpsPerBlock) {
        const int64_t row = (int64_t)touched[w] * M;
        split_one_cell<P>(cut + row, Q + row, C + row, m, nodes, parent, left, right, T, eps, max_iter, n_nodes,
                          status, s_q[warp], s_c[warp], s_cut[warp], s_nc[warp], s_b[warp]);
    }
}


// ---------------------------------------------------------------- bucketed learning
// counters (rll_grid::n_touched): [0] touched cells, [1] bucket space claimed,
// [2] cells for the sorting block path, [3] cells for the grouping block path;
// rll_grid::big lists the latter, rll_grid::big + H the former
constexpr int kBucketThreads = 256;
constexpr int kTilesPerWarp = 4;         // 32-record tiles one warp counts / scatters
constexpr uint32_t kWarpBucket = 240;    // records of a cell one warp orders in shared memory
constexpr uint32_t kBlockGroup = 1024;   // records of a cell one block orders by grouping and ranking
constexpr int kGroupThreads = 256;
constexpr uint32_t kBlockSort = 8192;    // records of a cell one block sorts in shared memory (power of 2)
constexpr size_t kBigSmem = kBlockSort * (sizeof(unsigned long long) + sizeof(uint32_t));
constexpr int kBigThreads = 512;

// 1. record counts per cell; the first adder appends the cell to the touched
// list. Each warp takes kTilesPerWarp tiles of 32 consecutive records.
__global__ void __launch_bounds__(kBucketThreads)
k_bucket_count(const uint32_t* __restrict__ rec_key, int64_t n, uint32_t HM, uint32_t M, uint32_t* __restrict__ cursor,
               uint32_t* __restrict__ touched, uint32_t* __restrict__ ctr)
{
    const int lane = threadIdx.x & 31;
    const int64_t tile0 = ((int64_t)blockIdx.x * (kBucketThreads / 32) + (threadIdx.x >> 5)) * kTilesPerWarp;
    uint32_t slot[kTilesPerWarp], peers[kTilesPerWarp], old[kTilesPerWarp];
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        const int64_t i = (tile0 + u) * 32 + lane;
        const uint32_t key = i < n ? __ldg(rec_key + i) : 0xFFFFFFFFu;
        slot[u] = key < HM ? key / M : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) peers[u] = __match_any_sync(0xffffffffu, slot[u]);
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        old[u] = 1u;
        if (slot[u] != 0xFFFFFFFFu && lane == __ffs(peers[u]) - 1)
            old[u] = atomicAdd(cursor + slot[u], (uint32_t)__popc(peers[u]));
    }
    // cells this lane saw first: one append per warp for all of them
    uint32_t fresh = 0;
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) fresh += old[u] == 0u;
    uint32_t x = fresh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    uint32_t base = 0;
    if (lane == 31 && x) base = atomicAdd(ctr, x);
    base = __shfl_sync(0xffffffffu, base, 31) + x - fresh;
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u)
        if (old[u] == 0u) touched[base++] = slot[u];
}

// 2. one contiguous bucket per touched cell (one atomic per warp)
__global__ void __launch_bounds__(kBucketThreads)
k_bucket_claim(const uint32_t* __restrict__ touched, uint32_t* __restrict__ ctr, uint32_t* __restrict__ cursor,
               uint32_t* __restrict__ start, uint32_t* __restrict__ len)
{
    const uint32_t total = *(volatile uint32_t*)ctr;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < total; w += warps) {
        const uint32_t c = w * 32 + lane;
        const uint32_t slot = c < total ? touched[c] : 0u;
        const uint32_t cnt = c < total ? cursor[slot] : 0u;
        uint32_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        uint32_t base = 0;
        if (lane == 31) base = atomicAdd(ctr + 1, x);
        base = __shfl_sync(0xffffffffu, base, 31);
        if (c < total) {
            start[c] = base + x - cnt;
            len[c] = cnt;
            cursor[slot] = base + x - cnt;
        }
    }
}

// 3. every record to its cell's bucket: sample id, cluster and reward (a
// warp's lanes that share a cell take consecutive places; the order inside a
// bucket depends on scheduling and is restored by the per-cell ordering)
// Bucket entry of a record: sample id, cluster, reward bits (three arrays)
struct Bucket {
    uint32_t* sid;
    uint8_t* s;
    uint32_t* val;
};

__global__ void __launch_bounds__(kBucketThreads)
k_bucket_scatter(const uint32_t* __restrict__ rec_key, const float* __restrict__ rec_val, int64_t n, uint32_t HM,
                 uint32_t M, uint32_t* __restrict__ cursor, Bucket bucket)
{
    const int lane = threadIdx.x & 31;
    const int64_t tile0 = ((int64_t)blockIdx.x * (kBucketThreads / 32) + (threadIdx.x >> 5)) * kTilesPerWarp;
    uint32_t slot[kTilesPerWarp], clus[kTilesPerWarp], val[kTilesPerWarp], peers[kTilesPerWarp],
        base[kTilesPerWarp];
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        const int64_t i = (tile0 + u) * 32 + lane;
        const uint32_t key = i < n ? __ldg(rec_key + i) : 0xFFFFFFFFu;
        val[u] = i < n ? __float_as_uint(__ldg(rec_val + i)) : 0u;
        slot[u] = key < HM ? key / M : 0xFFFFFFFFu;
        clus[u] = key < HM ? key % M : 0u;
    }
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) peers[u] = __match_any_sync(0xffffffffu, slot[u]);
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        base[u] = 0u;
        if (slot[u] != 0xFFFFFFFFu && lane == __ffs(peers[u]) - 1)
            base[u] = atomicAdd(cursor + slot[u], (uint32_t)__popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        const uint32_t b = __shfl_sync(0xffffffffu, base[u], __ffs(peers[u]) - 1);
        if (slot[u] != 0xFFFFFFFFu) {
            const uint32_t d = b + __popc(peers[u] & lanemask_lt());
            bucket.sid[d] = (uint32_t)((tile0 + u) * 32 + lane);
            bucket.s[d] = (uint8_t)clus[u];
            bucket.val[d] = val[u];
        }
    }
}

// Shared arrays of one team (a warp or a block) ordering one cell's records:
// A = bucket order, then (cluster, sample) order; B = grouped by cluster,
// then the cdf scratch.
template <uint32_t CAP>
struct CellOrder {
    uint32_t a_sid[CAP];
    uint32_t a_val[CAP];
    uint32_t b_sid[CAP];
    uint32_t b_val[CAP];
    uint8_t a_s[CAP];
    uint8_t b_s[CAP];
    uint32_t start[kMaxCut];  // first position of each cluster in B
    uint32_t cur[kMaxCut];    // scatter cursors, then one past the last position
    float q[kMaxCut];
};

// A team orders one cell; its first warp (lead()) also scans and composes.
struct WarpTeam {
    __device__ __forceinline__ uint32_t tid() const { return threadIdx.x & 31; }
    __device__ __forceinline__ uint32_t size() const { return 32; }
    __device__ __forceinline__ bool lead() const { return true; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};
struct BlockTeam {
    __device__ __forceinline__ uint32_t tid() const { return threadIdx.x; }
    __device__ __forceinline__ uint32_t size() const { return blockDim.x; }
    __device__ __forceinline__ bool lead() const { return threadIdx.x < 32; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

template <int P>
__device__ __forceinline__ void load_q_row(const typename Store<P>::T* qrow, uint32_t m, float* q)
{
    for (uint32_t s = threadIdx.x & 31; s < m; s += 32) q[s] = Store<P>::load(qrow[s]);
}

template <int P>
__device__ __forceinline__ void store_q_row(typename Store<P>::T* qrow, uint32_t m, float* q)
{
    for (uint32_t s = threadIdx.x & 31; s < m; s += 32) {
        const typename Store<P>::T st = Store<P>::store(q[s]);
        qrow[s] = st;
        q[s] = Store<P>::load(st);
    }
}

// Eq. 1 + Eq. 2 of one cell from its bucket of nr <= CAP records: grouped
// by cluster (counting sort, any order inside a group), then each record's
// rank by sample id inside its group is counted, which puts them in
// (cluster, sample) order; warp 0 of the team composes, stores Q and
// rebuilds C. Called by every thread of the team.
template <int P, uint32_t CAP, class Team>
__device__ void learn_cell_grouped(Team team, CellOrder<CAP>& o, const uint32_t* __restrict__ bsid,
                                   const uint8_t* __restrict__ bs, const uint32_t* __restrict__ bval, uint32_t nr,
                                   uint32_t M, uint32_t m, float alpha, float eps, typename Store<P>::T* qrow,
                                   typename Store<P>::T* crow, uint32_t* status)
{
    const uint32_t t = team.tid(), T = team.size();
    const int lane = threadIdx.x & 31;
    const bool w0 = team.lead();
    for (uint32_t s = t; s < M; s += T) o.start[s] = 0u;
    if (w0) load_q_row<P>(qrow, m, o.q);
    team.sync();
    for (uint32_t k = t; k < nr; k += T) {
        const uint32_t s = bs[k];
        o.a_sid[k] = bsid[k];
        o.a_val[k] = bval[k];
        o.a_s[k] = (uint8_t)s;
        atomicAdd(&o.start[s], 1u);
    }
    team.sync();
    if (w0) {  // cluster starts: exclusive scan over M bins, ipl consecutive bins a lane
        const uint32_t ipl = (M + 31) >> 5, lo = lane * ipl, hi = min(M, lo + ipl);
        uint32_t sum = 0;
        for (uint32_t s = lo; s < hi; ++s) sum += o.start[s];
        uint32_t y = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += v;
        }
        uint32_t run = y - sum;
        for (uint32_t s = lo; s < hi; ++s) {
            const uint32_t c = o.start[s];
            o.start[s] = run;
            o.cur[s] = run;
            run += c;
        }
    }
    team.sync();
    for (uint32_t k = t; k < nr; k += T) {
        const uint32_t s = o.a_s[k];
        const uint32_t d = atomicAdd(&o.cur[s], 1u);
        if (d >= nr) {  // impossible unless the counts are corrupt: flag, skip the write
            atomicOr(status, (uint32_t)RLL_E_DEVICE);
            continue;
        }
        o.b_sid[d] = o.a_sid[k];
        o.b_val[d] = o.a_val[k];
        o.b_s[d] = (uint8_t)s;
    }
    team.sync();
    for (uint32_t k = t; k < nr; k += T) {
        const uint32_t s = o.b_s[k], sid = o.b_sid[k];
        const uint32_t lo = o.start[s], hi = o.cur[s];
        const uint32_t end = min(hi, nr);
        uint32_t rank = 0, j = lo;
        for (; j + 4 <= end; j += 4) {
            const uint32_t x0 = o.b_sid[j], x1 = o.b_sid[j + 1], x2 = o.b_sid[j + 2], x3 = o.b_sid[j + 3];
            rank += (x0 < sid) + (x1 < sid) + (x2 < sid) + (x3 < sid);
        }
        for (; j < end; ++j) rank += o.b_sid[j] < sid;
        if (lo + rank >= nr) {
            atomicOr(status, (uint32_t)RLL_E_DEVICE);
            continue;
        }
        o.a_s[lo + rank] = (uint8_t)s;
        o.a_val[lo + rank] = o.b_val[k];
    }
    team.sync();
    if (T == 32) {
        learn_records<P>([&](uint32_t j) { return make_uint2(o.a_s[j], o.a_val[j]); }, nr, m, alpha, o.q);
    } else {  // a block: warp w composes the groups of clusters w, w + warps, ...
        const uint32_t warps = T >> 5;
        for (uint32_t s = threadIdx.x >> 5; s < M; s += warps) {
            const uint32_t lo = o.start[s], hi = o.cur[s];
            if (hi > lo)
                learn_records<P>([&](uint32_t j) { return make_uint2(o.a_s[lo + j], o.a_val[lo + j]); }, hi - lo,
                                 m, alpha, o.q);
        }
        team.sync();
    }
    if (w0) {
        store_q_row<P>(qrow, m, o.q);
        __syncwarp();
        warp_rebuild_cdf<P>(o.q, (int)m, eps, crow, reinterpret_cast<float*>(o.b_sid),
                            reinterpret_cast<uint16_t*>(o.b_val));
    }
}

// 4. one warp per cell of a list (list == nullptr: every touched cell) with
// at most CAP records; a larger cell is appended to the next list (`next`,
// its count at *next_count) for the block path.
template <int P, uint32_t CAP, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
k_learn_tier(const Bucket bucket, const uint32_t* __restrict__ list, const uint32_t* __restrict__ list_count,
             uint32_t* __restrict__ next, uint32_t* __restrict__ next_count, const uint32_t* __restrict__ touched,
             const uint32_t* __restrict__ start, const uint32_t* __restrict__ len, uint32_t* __restrict__ cursor,
             uint32_t M, uint32_t m, typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C,
             float alpha, float eps, uint32_t* __restrict__ status)
{
    __shared__ CellOrder<CAP> rows[WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t total = *(volatile const uint32_t*)list_count;
    for (uint32_t i = blockIdx.x * WARPS + warp; i < total; i += gridDim.x * WARPS) {
        const uint32_t w = list ? list[i] : i;
        const uint32_t slot = touched[w], nr = len[w];
        if (nr > CAP) {
            if (lane == 0) next[atomicAdd(next_count, 1u)] = w;
            continue;
        }
        const int64_t row = (int64_t)slot * M;
        const uint32_t b0 = start[w];
        learn_cell_grouped<P>(WarpTeam{}, rows[warp], bucket.sid + b0, bucket.s + b0, bucket.val + b0, nr, M, m,
                              alpha, eps, Q + row, C + row, status);
        if (lane == 0) cursor[slot] = 0u;
    }
}

// Eq. 1 of one cell whose records are sorted by (cluster, sample id), by a
// whole block: cluster s occupies positions gs[s] .. ge[s]; cls(j) is the
// cluster and val(j) the reward bits of record j. Warp w composes clusters
// w, w + warps, ... (disjoint Q entries). All threads of the block call it.
template <int P, class Cls, class Val>
__device__ void compose_sorted_block(Cls cls, Val val, uint32_t nr, uint32_t M, uint32_t m, float alpha, float* q,
                                     uint32_t* gs, uint32_t* ge)
{
    for (uint32_t s = threadIdx.x; s < M; s += blockDim.x) gs[s] = ge[s] = 0u;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nr; j += blockDim.x) {
        const uint32_t s = cls(j);
        if (s >= M) continue;
        if (j == 0 || cls(j - 1) != s) gs[s] = j;
        if (j + 1 == nr || cls(j + 1) != s) ge[s] = j + 1;
    }
    __syncthreads();
    const uint32_t warps = blockDim.x >> 5;
    for (uint32_t s = threadIdx.x >> 5; s < M; s += warps) {
        const uint32_t lo = gs[s], hi = ge[s];
        if (hi > lo) learn_records<P>([&](uint32_t j) { return make_uint2(s, val(lo + j)); }, hi - lo, m, alpha, q);
    }
    __syncthreads();
}

// 5a. one block per cell of the grouping list (up to kBlockGroup records):
// the ordering of the warp path done by the whole block, warps composing
// different clusters in parallel; larger cells go to the sorting list.
template <int P>
__global__ void __launch_bounds__(kGroupThreads)
k_learn_group(const Bucket bucket, uint32_t* __restrict__ ctr, const uint32_t* __restrict__ touched,
              const uint32_t* __restrict__ start, const uint32_t* __restrict__ len, const uint32_t* __restrict__ list,
              uint32_t* __restrict__ next, uint32_t* __restrict__ cursor, uint32_t M, uint32_t m,
              typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C, float alpha, float eps,
              uint32_t* __restrict__ status)
{
    __shared__ CellOrder<kBlockGroup> o;
    const uint32_t n = *(volatile const uint32_t*)(ctr + 3);
    for (uint32_t bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const uint32_t w = list[bi];
        const uint32_t slot = touched[w], b0 = start[w], nr = len[w];
        if (nr > kBlockGroup) {
            if (threadIdx.x == 0) next[atomicAdd(ctr + 2, 1u)] = w;
            continue;  // uniform across the block
        }
        const int64_t row = (int64_t)slot * M;
        learn_cell_grouped<P>(BlockTeam{}, o, bucket.sid + b0, bucket.s + b0, bucket.val + b0, nr, M, m, alpha, eps,
                              Q + row, C + row, status);
        if (threadIdx.x == 0) cursor[slot] = 0u;
        __syncthreads();
    }
}

// 5b. one block per cell of the sorting list. Up to kBlockSort records: keys
// cluster << 45 | sample id << 13 | bucket index sorted by a bitonic network
// in shared memory, rewards gathered in that order. Larger cells: (cluster
// << 32 | sample id) sorted in place in global scratch, rewards read by
// sample id. Then Eq. 1 (warps composing different clusters) and Eq. 2.
template <int P>
__global__ void __launch_bounds__(kBigThreads)
k_learn_big(const Bucket bucket, unsigned long long* __restrict__ wide, const float* __restrict__ rec_val,
            const uint32_t* __restrict__ ctr,
            const uint32_t* __restrict__ touched, const uint32_t* __restrict__ start,
            const uint32_t* __restrict__ len, const uint32_t* __restrict__ big, uint32_t* __restrict__ cursor,
            uint32_t M, uint32_t m, typename Store<P>::T* __restrict__ Q, typename Store<P>::T* __restrict__ C,
            float alpha, float eps, uint32_t* __restrict__ status)
{
    extern __shared__ unsigned long long s_key[];      // kBlockSort keys, then kBlockSort rewards (u32)
    uint32_t* s_val = reinterpret_cast<uint32_t*>(s_key + kBlockSort);
    __shared__ float s_q[kMaxCut], s_c[kMaxCut];
    __shared__ uint16_t s_b[kMaxCut];
    __shared__ uint32_t s_gs[kMaxCut], s_ge[kMaxCut];
    const uint32_t n_big = *(volatile const uint32_t*)(ctr + 2);
    for (uint32_t bi = blockIdx.x; bi < n_big; bi += gridDim.x) {
        const uint32_t w = big[bi];
        const uint32_t slot = touched[w], b0 = start[w], nr = len[w];
        const int64_t row = (int64_t)slot * M;
        if (threadIdx.x < 32) load_q_row<P>(Q + row, m, s_q);
        if (nr <= kBlockSort) {
            for (uint32_t k = threadIdx.x; k < nr; k += blockDim.x)
                s_key[k] = ((unsigned long long)bucket.s[b0 + k] << 45) |
                           ((unsigned long long)bucket.sid[b0 + k] << 13) | k;
            __syncthreads();
            bitonic_sort_u64(s_key, nr, threadIdx.x, blockDim.x, BlockSync{});
            for (uint32_t j = threadIdx.x; j < nr; j += blockDim.x)
                s_val[j] = bucket.val[b0 + (uint32_t)(s_key[j] & (kBlockSort - 1))];
            __syncthreads();
            compose_sorted_block<P>([&](uint32_t j) { return (uint32_t)(s_key[j] >> 45); },
                                    [&](uint32_t j) { return s_val[j]; }, nr, M, m, alpha, s_q, s_gs, s_ge);
        } else {
            unsigned long long* rec = wide + b0;
            for (uint32_t k = threadIdx.x; k < nr; k += blockDim.x)
                rec[k] = ((unsigned long long)bucket.s[b0 + k] << 32) | bucket.sid[b0 + k];
            __syncthreads();
            bitonic_sort_u64(rec, nr, threadIdx.x, blockDim.x, BlockSync{});
            for (uint32_t k = threadIdx.x; k < nr; k += blockDim.x) {
                const unsigned long long e = rec[k];
                rec[k] = (e & 0xFFFFFFFF00000000ull) | __float_as_uint(__ldg(rec_val + (uint32_t)e));
            }
            __syncthreads();
            compose_sorted_block<P>([&](uint32_t j) { return (uint32_t)(rec[j] >> 32); },
                                    [&](uint32_t j) { return (uint32_t)rec[j]; }, nr, M, m, alpha, s_q, s_gs, s_ge);
        }
        if (threadIdx.x < 32) {
            store_q_row<P>(Q + row, m, s_q);
            __syncwarp();
            warp_rebuild_cdf<P>(s_q, (int)m, eps, C + row, s_c, s_b);
            if (threadIdx.x == 0) cursor[slot] = 0u;
        }
        __syncthreads();
    }
}

// k_learn_big's shared-memory opt-in (above the 48 KB default), once per
// device and precision
template <int P>
cudaError_t big_smem_attribute(int device)
{
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device >= 0 && device < 64 && done[device]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_learn_big<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kBigSmem);
    if (e == cudaSuccess && device >= 0 && device < 64) done[device] = true;
    return e;
}

template <int P>
int learn_t(rll_ctx* ctx, rll_grid* g, const uint32_t* rec_key, const float* rec_val, int64_t n)
{
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemsetAsync(g->n_touched, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "memset touched");
    if (n <= 0) return RLL_OK;
    if (n > 0xFFFFFFFFll) return fail(ctx, RLL_E_INVALID, "more than 2^32 - 1 records");
    if (g->cursor_dirty) {
        e = cudaMemsetAsync(g->cursor, 0, 4 * (size_t)g->H, s);
        if (e != cudaSuccess) return check_cuda(ctx, e, "memset cursors");
        g->cursor_dirty = false;
    }
    const uint32_t HM = g->H * g->M;
    // scratch per record: bucket sample id (4 B), reward (4 B), cluster (1 B),
    // and the block path's in-place sort buffer (8 B, used only by cells
    // above kBlockSort records)
    const size_t n4 = ((size_t)n * 4 + 255) & ~(size_t)255, n1 = ((size_t)n + 255) & ~(size_t)255;
    char* ws = static_cast<char*>(ws_get(ctx, 2 * n4 + n1 + 8 * (size_t)n));
    if (!ws) return RLL_E_NOMEM;
    Bucket bucket{reinterpret_cast<uint32_t*>(ws), reinterpret_cast<uint8_t*>(ws + 2 * n4),
                  reinterpret_cast<uint32_t*>(ws + n4)};
    auto* wide = reinterpret_cast<unsigned long long*>(ws + 2 * n4 + n1);
    const int64_t per_block = (int64_t)kBucketThreads * kTilesPerWarp;
    const unsigned rblocks = (unsigned)((n + per_block - 1) / per_block);
    const int sms = device_sm_count(g->device);
    using T = typename Store<P>::T;
    g->cursor_dirty = true;
    k_bucket_count<<<rblocks, kBucketThreads, 0, s>>>(rec_key, n, HM, g->M, g->cursor, g->touched, g->n_touched);
    k_bucket_claim<<<sms * 2, kBucketThreads, 0, s>>>(g->touched, g->n_touched, g->cursor, g->touched_start,
                                                     g->touched_len);
    k_bucket_scatter<<<rblocks, kBucketThreads, 0, s>>>(rec_key, rec_val, n, HM, g->M, g->cursor, bucket);
    uint32_t* group_list = g->big;
    uint32_t* sort_list = g->big + g->H;
    k_learn_tier<P, kWarpBucket, 6, 5><<<sms * 5, 6 * 32, 0, s>>>(
        bucket, nullptr, g->n_touched, group_list, g->n_touched + 3, g->touched, g->touched_start, g->touched_len,
        g->cursor, g->M, g->m, (T*)g->Q, (T*)g->C, g->p.alpha, g->p.eps, ctx->d_status);
    k_learn_group<P><<<sms * 4, kGroupThreads, 0, s>>>(bucket, g->n_touched, g->touched, g->touched_start,
                                                        g->touched_len, group_list, sort_list, g->cursor, g->M, g->m,
                                                        (T*)g->Q, (T*)g->C, g->p.alpha, g->p.eps, ctx->d_status);
    e = big_smem_attribute<P>(g->device);
    if (e != cudaSuccess) return check_cuda(ctx, e, "learn: shared memory opt-in");
    k_learn_big<P><<<sms * 2, kBigThreads, kBigSmem, s>>>(bucket, wide, rec_val, g->n_touched, g->touched,
                                                          g->touched_start, g->touched_len, sort_list, g->cursor,
                                                          g->M, g->m, (T*)g->Q, (T*)g->C, g->p.alpha, g->p.eps,
                                                          ctx->d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(ctx, e, "learn kernels");
    g->cursor_dirty = false;
    return RLL_OK;
}

template <int P>
int split_t(rll_ctx* ctx, rll_grid* g, const rll_tree* t)
{
    using T = typename Store<P>::T;
    const int blocks = device_sm_count(g->device) * 8;
    k_split<P><<<blocks, kWarpsPerBlock * 32, 0, ctx->stream>>>(g->M, g->m, g->touched, g->n_touched, g->cut,
                                                                  (T*)g->Q, (T*)g->C, t->nodes, t->parent, t->left,
                                                                  t->right, g->p.threshold, g->p.eps,
                                                                  split_steps(g->p), 2 * t->n - 1, ctx->d_status);
    return check_cuda(ctx, cudaGetLastError(), "split kernel");
}

template <int P>
int init_t(rll_ctx* ctx, rll_grid* g)
{
    using T = typename Store<P>::T;
    cudaStream_t s = ctx->stream;
    k_default_row<P><<<1, 32, 0, s>>>(g->m, g->p.q_init, g->p.eps, (T*)g->def_Q, (T*)g->def_C);
    const int64_t total = (int64_t)g->H * g->M;
    k_fill_rows<P><<<device_sm_count(g->device) * 4, 256, 0, s>>>(total, g->M, g->m, g->def_cut, (const T*)g->def_Q,
                                                                  (const T*)g->def_C, g->cut, (T*)g->Q, (T*)g->C);
    return check_cuda(ctx, cudaGetLastError(), "grid init");
}

}  // namespace

int key_bits(uint64_t hm_plus_one)
{
    int b = 0;
    while ((1ull << b) < hm_plus_one) ++b;
    return b;
}

int device_sm_count(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

int grid_init(rll_ctx* ctx, rll_grid* g)
{
    switch (g->p.precision) {
    case RLL_PREC_FP16: return init_t<RLL_PREC_FP16>(ctx, g);
    case RLL_PREC_BF16: return init_t<RLL_PREC_BF16>(ctx, g);
    default: return init_t<RLL_PREC_FP32>(ctx, g);
    }
}

int grid_to_float(rll_ctx* ctx, const rll_grid* g, float* q, float* c)
{
    const int64_t total = (int64_t)g->H * g->M;
    const unsigned blocks = device_sm_count(g->device) * 4;
    switch (g->p.precision) {
    case RLL_PREC_FP16:
        k_to_float<RLL_PREC_FP16><<<blocks, 256, 0, ctx->stream>>>(total, (const __half*)g->Q, (const __half*)g->C, q, c);
        break;
    case RLL_PREC_BF16:
        k_to_float<RLL_PREC_BF16><<<blocks, 256, 0, ctx->stream>>>(total, (const __nv_bfloat16*)g->Q,
                                                                   (const __nv_bfloat16*)g->C, q, c);
        break;
    default:
        k_to_float<RLL_PREC_FP32><<<blocks, 256, 0, ctx->stream>>>(total, (const float*)g->Q, (const float*)g->C, q, c);
    }
    return check_cuda(ctx, cudaGetLastError(), "grid export");
}

template <int P>
void from_float_t(rll_ctx* ctx, rll_grid* g, const float* q, const float* c)
{
    using T = typename Store<P>::T;
    const int64_t total = (int64_t)g->H * g->M;
    const unsigned blocks = device_sm_count(g->device) * 4;
    k_from_float<P><<<blocks, 256, 0, ctx->stream>>>(total, q, c, (T*)g->Q, (T*)g->C);
    k_reset_empty_rows<P><<<blocks, 256, 0, ctx->stream>>>(total, g->M, g->m, g->keys, g->def_cut, (const T*)g->def_Q,
                                                           (const T*)g->def_C, g->cut, (T*)g->Q, (T*)g->C);
}

int grid_from_float(rll_ctx* ctx, rll_grid* g, const float* q, const float* c)
{
    switch (g->p.precision) {
    case RLL_PREC_FP16: from_float_t<RLL_PREC_FP16>(ctx, g, q, c); break;
    case RLL_PREC_BF16: from_float_t<RLL_PREC_BF16>(ctx, g, q, c); break;
    default: from_float_t<RLL_PREC_FP32>(ctx, g, q, c);
    }
    return check_cuda(ctx, cudaGetLastError(), "grid import");
}

void launch_cell_heads(cudaStream_t s, const uint32_t* sk, int64_t n, uint32_t HM, uint32_t M, uint32_t* touched,
                       uint32_t* touched_start, uint32_t* n_touched)
{
    if (n <= 0) return;
    k_cell_heads<<<(unsigned)((n + 256 * kHeadItems - 1) / (256 * kHeadItems)), 256, 0, s>>>(sk, n, HM, M, touched,
                                                                                           touched_start, n_touched);
}

int grid_mark_occupied(rll_ctx* ctx, rll_grid* g)
{
    cudaError_t e = cudaMemsetAsync(g->n_touched, 0, sizeof(uint32_t), ctx->stream);
    if (e != cudaSuccess) return check_cuda(ctx, e, "memset touched");
    k_mark_occupied<<<(g->H + 255) / 256, 256, 0, ctx->stream>>>(g->keys, g->H, g->touched, g->n_touched);
    return check_cuda(ctx, cudaGetLastError(), "mark occupied");
}

int learn_update(rll_ctx* ctx, rll_grid* g, const uint32_t* rec_key, const float* rec_val, int64_t n)
{
    switch (g->p.precision) {
    case RLL_PREC_FP16: return learn_t<RLL_PREC_FP16>(ctx, g, rec_key, rec_val, n);
    case RLL_PREC_BF16: return learn_t<RLL_PREC_BF16>(ctx, g, rec_key, rec_val, n);
    default: return learn_t<RLL_PREC_FP32>(ctx, g, rec_key, rec_val, n);
    }
}

int split_collapse(rll_ctx* ctx, rll_grid* g, const rll_tree* t)
{
    switch (g->p.precision) {
    case RLL_PREC_FP16: return split_t<RLL_PREC_FP16>(ctx, g, t);
    case RLL_PREC_BF16: return split_t<RLL_PREC_BF16>(ctx, g, t);
    default: return split_t<RLL_PREC_FP32>(ctx, g, t);
    }
}

}  // namespace rll

// ---------------------------------------------------------------------------
// Learning step with caller-provided scratch (used by the allocation-free
// entry point in noalloc.cu): the same kernels as learn_update, but the sort
// buffers live in `scratch` (scratch_bytes long) instead of the context's
// growable workspace, so nothing is allocated.
namespace rll {
namespace {

template <int P>
int learn_scratch_t(rll_ctx* ctx, rll_grid* g, const uint32_t* rec_key, const float* rec_val, int64_t n, void* scratch)
{
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemsetAsync(g->n_touched, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "memset touched");
    if (n <= 0) return RLL_OK;
    const uint32_t HM = g->H * g->M;
    uint32_t *sk, *sv;
    e = radix_sort_pairs(s, rec_key, reinterpret_cast<const uint32_t*>(rec_val), n, key_bits((uint64_t)HM + 1), HM,
                         scratch, &sk, &sv);
    if (e != cudaSuccess) return check_cuda(ctx, e, "radix sort (records)");
    k_cell_heads<<<(unsigned)((n + 256 * kHeadItems - 1) / (256 * kHeadItems)), 256, 0, s>>>(
        sk, n, HM, g->M, g->touched, g->touched_start, g->n_touched);
    const int blocks = device_sm_count(g->device) * 8;
    using T = typename Store<P>::T;
    k_learn_cells<P><<<blocks, kWarpsPerBlock * 32, 0, s>>>(sk, sv, n, HM, g->M, g->m, g->touched, g->touched_start,
                                                             g->n_touched, (T*)g->Q, (T*)g->C, g->p.alpha, g->p.eps);
    return check_cuda(ctx, cudaGetLastError(), "learn kernels");
}

}  // namespace

int learn_update_with_scratch(rll_ctx* ctx, rll_grid* g, const uint32_t* rec_key, const float* rec_val, int64_t n,
                              void* scratch, size_t scratch_bytes)
{
    if (n > 0 && radix_sort_scratch_bytes(n) > scratch_bytes)
        return fail(ctx, RLL_E_INVALID, "scratch too small for this many records");
    switch (g->p.precision) {
    case RLL_PREC_FP16: return learn_scratch_t<RLL_PREC_FP16>(ctx, g, rec_key, rec_val, n, scratch);
    case RLL_PREC_BF16: return learn_scratch_t<RLL_PREC_BF16>(ctx, g, rec_key, rec_val, n, scratch);
    default: return learn_scratch_t<RLL_PREC_FP32>(ctx, g, rec_key, rec_val, n, scratch);
    }
}

}  // namespace rll
