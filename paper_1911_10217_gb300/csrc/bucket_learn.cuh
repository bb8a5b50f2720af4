// Learning step on records bucketed by cell (Section 3, Eq. 1 and Eq. 2),
// shared by the single-grid entry point (learn.cu) and the batched form
// (batched.cu). A key decoder (valid / cell / cluster of a record key) and a
// row map (Q and C rows, cut size and length, alpha and eps of a cell) adapt
// it to either record layout. See learn.cu for the method notes.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "learn_core.cuh"
#include "rll_device.cuh"

namespace rll {
namespace {  // every translation unit that includes this header gets its own copies

// one cell's rows and learning parameters
template <int P>
struct RowRef {
    typename Store<P>::T* Q;
    typename Store<P>::T* C;
    uint32_t M, m;
    float alpha, eps;
};

// ---------------------------------------------------------------- bucketed learning
// counters ctr[8]: [0] touched cells, [1] bucket space claimed, [2] cells for
// the sorting block path, [3] cells for the two-warp path, [4] [5] [7] work
// counters of the block, warp and two-warp phases, [6] cells for the grouping
// block path; lists[2 * cells]: the grouping list (two-warp cells from the
// front, block cells from the back), then the sorting list
constexpr int kBucketThreads = 256;
constexpr int kTilesPerWarp = 4;         // 32-record tiles one warp counts / scatters
constexpr uint32_t kWarpBucket = 240;    // records of a cell one warp orders in shared memory
constexpr uint32_t kPairBucket = 512;    // records of a cell two warps order together
constexpr uint32_t kBlockGroup = 1024;   // records of a cell one block orders by grouping and ranking
constexpr uint32_t kBlockSort = 8192;    // records of a cell one block sorts in shared memory (power of 2)
constexpr size_t kBigSmem = kBlockSort * (sizeof(unsigned long long) + sizeof(uint32_t));
constexpr int kBigThreads = 512;

// 1. record counts per cell and each record's rank among its cell's records
// (the cell's count before its warp's group, plus the lanes of the group
// below it); the first adder of a cell appends it to the touched list, one
// append per block. Each warp takes kTilesPerWarp tiles of 32 consecutive
// records. The ranks follow arrival order; the per-cell ordering restores
// sample order.
template <class Dec>
__global__ void __launch_bounds__(kBucketThreads)
k_bucket_count(const uint32_t* __restrict__ rec_key, int64_t n, Dec dec, uint32_t* __restrict__ cursor,
               uint32_t* __restrict__ touched, uint32_t* __restrict__ ctr, uint32_t* __restrict__ rank)
{
    pdl_begin();
    __shared__ uint32_t s_warp[kBucketThreads / 32];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile0 = ((int64_t)blockIdx.x * (kBucketThreads / 32) + warp) * kTilesPerWarp;
    uint32_t slot[kTilesPerWarp], peers[kTilesPerWarp], old[kTilesPerWarp];
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        const int64_t i = (tile0 + u) * 32 + lane;
        const uint32_t key = i < n ? __ldg(rec_key + i) : 0xFFFFFFFFu;
        slot[u] = dec.valid(key) ? dec.cell(key) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) peers[u] = __match_any_sync(0xffffffffu, slot[u]);
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        old[u] = 1u;
        if (slot[u] != 0xFFFFFFFFu && lane == __ffs(peers[u]) - 1)
            old[u] = atomicAdd(cursor + slot[u], (uint32_t)__popc(peers[u]));
    }
    uint32_t fresh = 0;
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        const uint32_t b = __shfl_sync(0xffffffffu, old[u], __ffs(peers[u]) - 1);
        if (slot[u] != 0xFFFFFFFFu) rank[(tile0 + u) * 32 + lane] = b + __popc(peers[u] & lanemask_lt());
        fresh += old[u] == 0u;
    }
    // cells this block saw first: one append for all of them
    uint32_t x = fresh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < kBucketThreads / 32; ++w) {
            const uint32_t v = s_warp[w];
            s_warp[w] = tot;
            tot += v;
        }
        s_base = tot ? atomicAdd(ctr, tot) : 0u;
    }
    __syncthreads();
    if (!fresh) return;
    uint32_t base = s_base + s_warp[warp] + x - fresh;
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u)
        if (old[u] == 0u) touched[base++] = slot[u];
}

// 2. one contiguous bucket per touched cell (one atomic per warp)
__global__ void __launch_bounds__(kBucketThreads)
k_bucket_claim(const uint32_t* __restrict__ touched, uint32_t* __restrict__ ctr, uint32_t* __restrict__ cursor,
               uint32_t* __restrict__ start, uint32_t* __restrict__ len, uint32_t* __restrict__ group_list,
               uint32_t* __restrict__ sort_list, uint32_t cells)
{
    pdl_begin();
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
        // cells above one warp's capacity: to the two-warp list (front of the grouping list),
        // the block list (its back) or the sorting list
        const bool to_pair = c < total && cnt > kWarpBucket && cnt <= kPairBucket;
        const bool to_group = c < total && cnt > kPairBucket && cnt <= kBlockGroup;
        const bool to_sort = c < total && cnt > kBlockGroup;
        const uint32_t pm = __ballot_sync(0xffffffffu, to_pair);
        const uint32_t gm = __ballot_sync(0xffffffffu, to_group), sm = __ballot_sync(0xffffffffu, to_sort);
        uint32_t pb = 0, gb = 0, sb = 0;
        if (lane == 0 && pm) pb = atomicAdd(ctr + 3, (uint32_t)__popc(pm));
        if (lane == 0 && gm) gb = atomicAdd(ctr + 6, (uint32_t)__popc(gm));
        if (lane == 0 && sm) sb = atomicAdd(ctr + 2, (uint32_t)__popc(sm));
        pb = __shfl_sync(0xffffffffu, pb, 0);
        gb = __shfl_sync(0xffffffffu, gb, 0);
        sb = __shfl_sync(0xffffffffu, sb, 0);
        const uint32_t below = (1u << lane) - 1u;
        if (to_pair) group_list[pb + __popc(pm & below)] = c;
        if (to_group) group_list[cells - 1u - (gb + __popc(gm & below))] = c;
        if (to_sort) sort_list[sb + __popc(sm & below)] = c;
    }
}

// 3. every record to its cell's bucket, at the bucket start (the claim left it
// in the cell's cursor) plus the record's rank: sample id, cluster and reward;
// no atomics
// Bucket entry of a record: sample id, cluster, reward bits in one 8-byte
// word. Up to 2^24 records: cluster << 56 | sample id << 32 | reward bits (one
// store per record); above: sample id << 32 | reward bits, the cluster in a
// byte array beside it.
struct Bucket {
    unsigned long long* word;
    uint8_t* s;  // nullptr: the cluster is in the word
    __device__ __forceinline__ void put(uint32_t d, uint32_t id, uint32_t cls, uint32_t bits) const
    {
        if (!s) {
            word[d] = ((unsigned long long)(cls << 24 | id) << 32) | bits;
        } else {
            word[d] = ((unsigned long long)id << 32) | bits;
            s[d] = (uint8_t)cls;
        }
    }
    __device__ __forceinline__ void get(uint32_t d, uint32_t& id, uint32_t& cls, uint32_t& bits) const
    {
        const unsigned long long e = word[d];
        bits = (uint32_t)e;
        if (!s) {
            id = (uint32_t)(e >> 32) & 0xFFFFFFu;
            cls = (uint32_t)(e >> 56);
        } else {
            id = (uint32_t)(e >> 32);
            cls = s[d];
        }
    }
};

template <class Dec>
__global__ void __launch_bounds__(kBucketThreads)
k_bucket_scatter(const uint32_t* __restrict__ rec_key, const float* __restrict__ rec_val, int64_t n, Dec dec,
                 const uint32_t* __restrict__ cursor, const uint32_t* __restrict__ rank, Bucket bucket)
{
    pdl_begin();
    const int64_t i0 = (int64_t)blockIdx.x * kBucketThreads * kTilesPerWarp + threadIdx.x;
    uint32_t key[kTilesPerWarp], val[kTilesPerWarp], rk[kTilesPerWarp], at[kTilesPerWarp];
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        const int64_t i = i0 + (int64_t)u * kBucketThreads;
        key[u] = i < n ? __ldg(rec_key + i) : 0xFFFFFFFFu;
        val[u] = i < n ? __float_as_uint(__ldg(rec_val + i)) : 0u;
        rk[u] = i < n ? __ldg(rank + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) at[u] = dec.valid(key[u]) ? __ldg(cursor + dec.cell(key[u])) : 0u;
#pragma unroll
    for (int u = 0; u < kTilesPerWarp; ++u) {
        if (!dec.valid(key[u])) continue;
        bucket.put(at[u] + rk[u], (uint32_t)(i0 + (int64_t)u * kBucketThreads), dec.cluster(key[u]), val[u]);
    }
}

// Shared arrays of one team (a warp or a block) ordering one cell's records
// (at most CAP records, cut sizes up to CLUS): A = bucket order, then
// (cluster, sample) order; B = grouped by cluster, then the cdf scratch.
template <uint32_t CAP, uint32_t CLUS = kMaxCut>
struct CellOrder {
    uint32_t a_sid[CAP];
    uint32_t a_val[CAP];
    uint32_t b_sid[CAP];
    uint32_t b_val[CAP];
    uint8_t a_s[CAP];
    uint8_t b_s[CAP];
    uint32_t start[CLUS];  // first position of each cluster in B
    uint32_t cur[CLUS];    // scatter cursors, then one past the last position
    float q[CLUS];
    // Once Eq. 1 is composed, the record arrays (the first 16 CAP bytes) are
    // dead: they give the float and 16-bit scratch rows (CLUS entries each)
    // of Eq. 2 and split-collapse.
    static_assert(16u * CAP >= 6u * CLUS, "record arrays too small for the scratch rows");
    __device__ __forceinline__ float* scratch_c() { return reinterpret_cast<float*>(this); }
    __device__ __forceinline__ uint16_t* scratch_bits()
    {
        return reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(this) + 4 * CLUS);
    }
};

// Split-collapse policy of the learning kernels: NoSplit leaves it to a
// separate call; a policy with kOn = true runs it on each cell right after the
// cell's Eq. 1, before the one Eq. 2 rebuild. row(cell) gives the cell's cut
// row, its light tree, threshold T and step limit.
struct SplitRow {
    uint32_t* cut;
    const NodeRec* nodes;
    const int32_t *parent, *left, *right;
    float T;
    uint32_t max_iter;
    int64_t n_nodes;
};
struct NoSplit {
    static constexpr bool kOn = false;
    __device__ __forceinline__ SplitRow row(uint32_t) const { return SplitRow{}; }
};
// one grid: cut rows of M entries at cut + slot M
struct WithSplit {
    static constexpr bool kOn = true;
    uint32_t* cut;
    uint32_t M;
    const NodeRec* nodes;
    const int32_t *parent, *left, *right;
    float T;
    uint32_t max_iter;
    int64_t n_nodes;
    __device__ __forceinline__ SplitRow row(uint32_t slot) const
    {
        return SplitRow{cut + (int64_t)slot * M, nodes, parent, left, right, T, max_iter, n_nodes};
    }
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
// warps 2p and 2p + 1 of a block; named barrier 1 + p (0 is __syncthreads)
struct PairTeam {
    __device__ __forceinline__ uint32_t tid() const { return threadIdx.x & 63u; }
    __device__ __forceinline__ uint32_t size() const { return 64; }
    __device__ __forceinline__ bool lead() const { return (threadIdx.x & 63u) < 32u; }
    // immediate barrier ids (a register id would reserve all 16 barriers of the block)
    __device__ __forceinline__ void sync() const
    {
        switch (threadIdx.x >> 6) {
        case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
        case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
        default: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
        }
    }
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

// Last step of one cell, by one warp: Q (q, m entries) stored to the table
// precision (q then holds the stored values); with a split policy,
// split-collapse on those values and the rows it changed stored; then Eq. 2
// from the final Q. Scratch rows of kMaxCut entries: cs, nc, c, bits.
template <int P, class Split>
__device__ void finish_cell(const Split& sp, uint32_t slot, float* q, uint32_t m, float eps,
                            typename Store<P>::T* qrow, typename Store<P>::T* crow, uint32_t* cs, uint32_t* nc,
                            float* c, uint16_t* bits, uint32_t* status)
{
    store_q_row<P>(qrow, m, q);
    __syncwarp();
    if constexpr (Split::kOn) {
        const int lane = threadIdx.x & 31;
        const SplitRow r = sp.row(slot);
        if (load_cut_row(r.cut, cs, m, r.n_nodes, status)) {
            const uint32_t steps = split_collapse_steps<P>(cs, q, c, nc, m, r.nodes, r.parent, r.left, r.right, r.T,
                                                           r.max_iter, r.n_nodes);
            if (steps) {
                for (uint32_t s = lane; s < m; s += 32) {
                    r.cut[s] = cs[s];
                    qrow[s] = Store<P>::store(q[s]);  // exact: q holds table values
                }
                __syncwarp();
            }
        }
    }
    warp_rebuild_cdf<P>(q, (int)m, eps, crow, c, bits);
}

// Eq. 1 + Eq. 2 of one cell from its bucket of nr <= CAP records: grouped
// by cluster (counting sort, any order inside a group), then each record's
// rank by sample id inside its group is counted, which puts them in
// (cluster, sample) order; warp 0 of the team composes, stores Q and
// rebuilds C. Called by every thread of the team.
template <int P, uint32_t CAP, uint32_t CLUS, class Team, class Split>
__device__ void learn_cell_grouped(Team team, CellOrder<CAP, CLUS>& o, const Bucket& bucket, uint32_t b0, uint32_t nr,
                                   uint32_t M, uint32_t m, float alpha, float eps, typename Store<P>::T* qrow,
                                   typename Store<P>::T* crow, const Split& sp, uint32_t slot, uint32_t* status)
{
    const uint32_t t = team.tid(), T = team.size();
    const int lane = threadIdx.x & 31;
    const bool w0 = team.lead();
    for (uint32_t s = t; s < M; s += T) o.start[s] = 0u;
    if (w0) load_q_row<P>(qrow, m, o.q);
    team.sync();
    // the bucket, four records a thread in flight at once
    for (uint32_t k0 = t; k0 < nr; k0 += 4 * T) {
        uint32_t rs[4], rsid[4], rval[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t k = k0 + u * T;
            rs[u] = rsid[u] = rval[u] = 0u;
            if (k < nr) bucket.get(b0 + k, rsid[u], rs[u], rval[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t k = k0 + u * T;
            if (k < nr) {
                o.a_sid[k] = rsid[u];
                o.a_val[k] = rval[u];
                o.a_s[k] = (uint8_t)rs[u];
                atomicAdd(&o.start[rs[u]], 1u);
            }
        }
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
    } else {  // a block or a pair: warp w of the team composes the groups of clusters w, w + warps, ...
        const uint32_t warps = T >> 5;
        for (uint32_t s = t >> 5; s < M; s += warps) {
            const uint32_t lo = o.start[s], hi = o.cur[s];
            if (hi > lo)
                learn_records<P>([&](uint32_t j) { return make_uint2(o.a_s[lo + j], o.a_val[lo + j]); }, hi - lo,
                                 m, alpha, o.q);
        }
        team.sync();
    }
    if (w0)  // cluster starts and cursors are dead too: the cut scratch rows
        finish_cell<P>(sp, slot, o.q, m, eps, qrow, crow, o.start, o.cur, o.scratch_c(), o.scratch_bits(), status);
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

// 4. Eq. 1 + Eq. 2 of every touched cell of at most kBlockGroup records in
// one persistent launch. Phase 1: blocks take the cells of the block list
// (more than kPairBucket records; the ordering of the warp path done by the
// whole block, warps composing different clusters in parallel). Phase 2: the
// block's warp pairs take the cells of the two-warp list (kWarpBucket ..
// kPairBucket records), three cells per block at a time. Phase 3: warps take
// the touched cells one by one and order those of at most kWarpBucket records
// themselves. Every phase draws from an atomic work counter (ctr[4], ctr[7],
// ctr[5]), so the long cells start first and the teams that drew one join the
// next phase late instead of leaving a tail; a warp fetches its next cell
// index while it works on the current one. Shared memory: one slab per warp;
// a pair's arrays lie in its two warps' slabs, the block's across all.
template <uint32_t CLUS>
struct LearnSmem {
    static constexpr size_t kWarp = sizeof(CellOrder<kWarpBucket, CLUS>);
    static constexpr size_t kPairHalf = (sizeof(CellOrder<kPairBucket, CLUS>) + 1) / 2;
    static constexpr size_t kSlab = ((kWarp > kPairHalf ? kWarp : kPairHalf) + 15) & ~(size_t)15;
};

template <int P, int WARPS, int MINB, uint32_t CLUS, class Rows, class Split>
__global__ void __launch_bounds__(WARPS * 32, MINB)
k_learn_buckets(const Bucket bucket, uint32_t* __restrict__ ctr, const uint32_t* __restrict__ group_list,
                const uint32_t* __restrict__ touched, const uint32_t* __restrict__ start,
                const uint32_t* __restrict__ len, uint32_t* __restrict__ cursor, Rows rows, Split sp,
                uint32_t* __restrict__ status, uint32_t cells)
{
    pdl_begin();
    static_assert(WARPS == 6, "three warp pairs, named barriers 1 .. 3");
    using L = LearnSmem<CLUS>;
    static_assert(sizeof(CellOrder<kBlockGroup, CLUS>) <= WARPS * L::kSlab, "block arrays exceed the slabs");
    __shared__ __align__(16) unsigned char smem[WARPS * L::kSlab];
    __shared__ uint32_t s_next, s_pair[WARPS / 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t n_group = *(volatile const uint32_t*)(ctr + 6);
    const uint32_t n_pair = *(volatile const uint32_t*)(ctr + 3);
    const uint32_t total = *(volatile const uint32_t*)ctr;
    auto& block_order = *reinterpret_cast<CellOrder<kBlockGroup, CLUS>*>(smem);
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(ctr + 4, 1u);
        __syncthreads();
        const uint32_t bi = s_next;
        __syncthreads();
        if (bi >= n_group) break;  // uniform across the block
        const uint32_t w = group_list[cells - 1u - bi];
        const uint32_t slot = touched[w], b0 = start[w], nr = len[w];
        const RowRef<P> r = rows.row(slot);
        learn_cell_grouped<P>(BlockTeam{}, block_order, bucket, b0, nr, r.M, r.m,
                              r.alpha, r.eps, r.Q, r.C, sp, slot, status);
        if (threadIdx.x == 0) cursor[slot] = 0u;
        __syncthreads();
    }
    // every warp of the block has left phase 1: pairs of warps, each in its own two slabs
    {
        const PairTeam team;
        const int pair = warp >> 1;
        auto& pair_order = *reinterpret_cast<CellOrder<kPairBucket, CLUS>*>(smem + 2 * pair * L::kSlab);
        for (;;) {
            if (team.tid() == 0) s_pair[pair] = atomicAdd(ctr + 7, 1u);
            team.sync();
            const uint32_t pi = s_pair[pair];
            team.sync();
            if (pi >= n_pair) break;  // uniform across the pair
            const uint32_t w = group_list[pi];
            const uint32_t slot = touched[w], b0 = start[w], nr = len[w];
            const RowRef<P> r = rows.row(slot);
            learn_cell_grouped<P>(team, pair_order, bucket, b0, nr, r.M, r.m,
                                  r.alpha, r.eps, r.Q, r.C, sp, slot, status);
            if (team.tid() == 0) cursor[slot] = 0u;
            team.sync();
        }
    }
    // both warps of the pair have left phase 2: the shared memory is per warp now
    auto& warp_order = *reinterpret_cast<CellOrder<kWarpBucket, CLUS>*>(smem + warp * L::kSlab);
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(ctr + 5, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < total) {
        const uint32_t i = next;
        uint32_t ahead = 0;
        if (lane == 0) ahead = atomicAdd(ctr + 5, 1u);
        const uint32_t slot = touched[i], nr = len[i];
        if (nr <= kWarpBucket) {
            const RowRef<P> r = rows.row(slot);
            const uint32_t b0 = start[i];
            learn_cell_grouped<P>(WarpTeam{}, warp_order, bucket, b0, nr, r.M,
                                  r.m, r.alpha, r.eps, r.Q, r.C, sp, slot, status);
            if (lane == 0) cursor[slot] = 0u;
        }
        next = __shfl_sync(0xffffffffu, ahead, 0);
    }
}

// 5b. one block per cell of the sorting list. Up to kBlockSort records: keys
// cluster << 45 | sample id << 13 | bucket index sorted by a bitonic network
// in shared memory, rewards gathered in that order. Larger cells: (cluster
// << 32 | sample id) sorted in place in global scratch, rewards read by
// sample id. Then Eq. 1 (warps composing different clusters) and Eq. 2.
template <int P, class Rows, class Split>
__global__ void __launch_bounds__(kBigThreads)
k_learn_big(const Bucket bucket, unsigned long long* __restrict__ wide, const float* __restrict__ rec_val,
            const uint32_t* __restrict__ ctr,
            const uint32_t* __restrict__ touched, const uint32_t* __restrict__ start,
            const uint32_t* __restrict__ len, const uint32_t* __restrict__ big, uint32_t* __restrict__ cursor,
            Rows rows, Split sp, uint32_t* __restrict__ status)
{
    pdl_begin();
    extern __shared__ unsigned long long s_key[];      // kBlockSort keys, then kBlockSort rewards (u32)
    uint32_t* s_val = reinterpret_cast<uint32_t*>(s_key + kBlockSort);
    __shared__ float s_q[kMaxCut], s_c[kMaxCut];
    __shared__ uint16_t s_b[kMaxCut];
    __shared__ uint32_t s_gs[kMaxCut], s_ge[kMaxCut];
    const uint32_t n_big = *(volatile const uint32_t*)(ctr + 2);
    for (uint32_t bi = blockIdx.x; bi < n_big; bi += gridDim.x) {
        const uint32_t w = big[bi];
        const uint32_t slot = touched[w], b0 = start[w], nr = len[w];
        const RowRef<P> r = rows.row(slot);
        const uint32_t M = r.M, m = r.m;
        const float alpha = r.alpha;
        if (threadIdx.x < 32) load_q_row<P>(r.Q, m, s_q);
        if (nr <= kBlockSort) {
            for (uint32_t k = threadIdx.x; k < nr; k += blockDim.x) {
                uint32_t id, cls, bits;
                bucket.get(b0 + k, id, cls, bits);
                s_key[k] = ((unsigned long long)cls << 45) | ((unsigned long long)id << 13) | k;
            }
            __syncthreads();
            bitonic_sort_u64(s_key, nr, threadIdx.x, blockDim.x, BlockSync{});
            for (uint32_t j = threadIdx.x; j < nr; j += blockDim.x) {
                uint32_t id, cls, bits;
                bucket.get(b0 + (uint32_t)(s_key[j] & (kBlockSort - 1)), id, cls, bits);
                s_val[j] = bits;
            }
            __syncthreads();
            compose_sorted_block<P>([&](uint32_t j) { return (uint32_t)(s_key[j] >> 45); },
                                    [&](uint32_t j) { return s_val[j]; }, nr, M, m, alpha, s_q, s_gs, s_ge);
        } else {
            unsigned long long* rec = wide + b0;
            for (uint32_t k = threadIdx.x; k < nr; k += blockDim.x) {
                uint32_t id, cls, bits;
                bucket.get(b0 + k, id, cls, bits);
                rec[k] = ((unsigned long long)cls << 32) | id;
            }
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
        if (threadIdx.x < 32) {  // the cluster bounds are dead: the cut scratch rows
            finish_cell<P>(sp, slot, s_q, m, r.eps, r.Q, r.C, s_gs, s_ge, s_c, s_b, status);
            if (threadIdx.x == 0) cursor[slot] = 0u;
        }
        __syncthreads();
    }
}

// k_learn_big's shared-memory opt-in (above the 48 KB default), once per
// device and precision
template <int P, class Rows, class Split>
cudaError_t big_smem_attribute(int device)
{
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device >= 0 && device < 64 && done[device]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_learn_big<P, Rows, Split>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kBigSmem);
    if (e == cudaSuccess && device >= 0 && device < 64) done[device] = true;
    return e;
}

// scratch of launch_bucketed_learn for n records: 8-byte bucket entries,
// cluster bytes (above 2^24 records), and the record ranks and in-place sort
// buffer (8 B: the ranks until the scatter, then the sort keys of cells above
// kBlockSort records)
inline size_t bucketed_scratch_bytes(int64_t n)
{
    const size_t n4 = ((size_t)n * 4 + 255) & ~(size_t)255, n1 = ((size_t)n + 255) & ~(size_t)255;
    return 2 * n4 + n1 + 8 * (size_t)n;
}

// Enqueues the whole learning step for n >= 1 records (cut sizes up to
// max_cut), every kernel with the programmatic launch dependency (each waits
// for its predecessor first). The caller has zeroed ctr[0..7] on the stream
// and holds `cursor` [cells] at zero (left at zero again); touched, start,
// len [cells] and lists [2 * cells] are outputs and scratch. Counters: ctr[0]
// touched cells, [1] claimed records, [2] sorting list, [3] two-warp list,
// [6] block list, [4] [5] [7] work counters of k_learn_buckets.
template <int P, class Dec, class Rows, class Split = NoSplit>
cudaError_t launch_bucketed_learn(cudaStream_t s, int device, int sms, const uint32_t* rec_key,
                                  const float* rec_val, int64_t n, Dec dec, Rows rows, uint32_t cells,
                                  uint32_t* cursor, uint32_t* touched, uint32_t* start, uint32_t* len,
                                  uint32_t* ctr, uint32_t* lists, void* scratch, uint32_t* status,
                                  uint32_t max_cut, Split sp = Split{})
{
    const size_t n4 = ((size_t)n * 4 + 255) & ~(size_t)255, n1 = ((size_t)n + 255) & ~(size_t)255;
    char* ws = static_cast<char*>(scratch);
    // 8-byte entries in the first 2 n4 bytes; the cluster bytes after them once sample ids need
    // more than 24 bits
    Bucket bucket{reinterpret_cast<unsigned long long*>(ws),
                  n <= (int64_t)1 << 24 ? nullptr : reinterpret_cast<uint8_t*>(ws + 2 * n4)};
    auto* wide = reinterpret_cast<unsigned long long*>(ws + 2 * n4 + n1);
    const int64_t per_block = (int64_t)kBucketThreads * kTilesPerWarp;
    const unsigned rblocks = (unsigned)((n + per_block - 1) / per_block);
    uint32_t* group_list = lists;
    uint32_t* sort_list = lists + cells;
    // record ranks: the first 4 n bytes of the in-place sort buffer (dead until k_learn_big)
    uint32_t* rank = reinterpret_cast<uint32_t*>(wide);
    cudaError_t e0 = launch_pdl(k_bucket_count<Dec>, dim3(rblocks), dim3(kBucketThreads), 0, s, rec_key, n, dec,
                                cursor, touched, ctr, rank);
    if (e0 == cudaSuccess)
        e0 = launch_pdl(k_bucket_claim, dim3(sms * 2), dim3(kBucketThreads), 0, s, touched, ctr, cursor, start, len,
                        group_list, sort_list, cells);
    if (e0 == cudaSuccess)
        e0 = launch_pdl(k_bucket_scatter<Dec>, dim3(rblocks), dim3(kBucketThreads), 0, s, rec_key, rec_val, n, dec,
                        cursor, rank, bucket);
    if (e0 != cudaSuccess) return e0;
    // cuts of at most 64 leaves: per-cluster arrays of 64 entries (30.5 KB of shared memory per
    // block), 56 registers, 6 blocks per SM; larger cuts: 256 entries (44.4 KB), 5 blocks per SM
    if (max_cut <= 64)
        e0 = launch_pdl(k_learn_buckets<P, 6, 6, 64, Rows, Split>, dim3(sms * 6), dim3(6 * 32), 0, s, bucket, ctr,
                        group_list, touched, start, len, cursor, rows, sp, status, cells);
    else
        e0 = launch_pdl(k_learn_buckets<P, 6, 5, kMaxCut, Rows, Split>, dim3(sms * 5), dim3(6 * 32), 0, s, bucket,
                        ctr, group_list, touched, start, len, cursor, rows, sp, status, cells);
    if (e0 != cudaSuccess) return e0;
    cudaError_t e = big_smem_attribute<P, Rows, Split>(device);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_learn_big<P, Rows, Split>, dim3(sms * 2), dim3(kBigThreads), kBigSmem, s, bucket, wide,
                      rec_val, ctr, touched, start, len, sort_list, cursor, rows, sp, status);
}

}  // namespace
}  // namespace rll
