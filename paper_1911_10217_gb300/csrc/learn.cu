// End-of-pass learning (Section 3, Eq. 1 and Eq. 2) and split-collapse
// (Section 3, Fig. "TreeCuts"; Section 3.1).
//
// learn_update (records bucketed by cell, then sorted per cell):
//   1. count: one thread per record; the lanes of a warp that hold the same
//      cell add their count with one atomic on the cell's cursor, each record
//      keeps its rank among the cell's records (the returned count plus its
//      place among the warp's lanes), and the first adder of a cell appends
//      it to the touched-cell list (one append per block);
//   2. claim: every touched cell takes a contiguous bucket of its record
//      count (one atomic per warp) and its cursor becomes the bucket start;
//   3. scatter: every record goes to its bucket start plus its rank (sample
//      id, cluster, reward; one 8-byte word while sample ids fit 24 bits);
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
// restores sample order, so the result is deterministic. Every kernel of the
// step is launched with the programmatic launch dependency (launch_pdl).
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

#include "bucket_learn.cuh"
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


// record key slot * M + cluster of one grid
struct GridDec {
    uint32_t HM, M;
    __device__ __forceinline__ bool valid(uint32_t k) const { return k < HM; }
    __device__ __forceinline__ uint32_t cell(uint32_t k) const { return k / M; }
    __device__ __forceinline__ uint32_t cluster(uint32_t k) const { return k % M; }
};

// rows of one grid
template <int P>
struct GridRows {
    typename Store<P>::T* Q;
    typename Store<P>::T* C;
    uint32_t M, m;
    float alpha, eps;
    __device__ __forceinline__ RowRef<P> row(uint32_t cell) const
    {
        const int64_t r = (int64_t)cell * M;
        return RowRef<P>{Q + r, C + r, M, m, alpha, eps};
    }
};

template <int P, class Split = NoSplit>
int learn_t(rll_ctx* ctx, rll_grid* g, const uint32_t* rec_key, const float* rec_val, int64_t n, Split sp = Split{})
{
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemsetAsync(g->n_touched, 0, 8 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "memset touched");
    if (n <= 0) return RLL_OK;
    if (n > 0xFFFFFFFFll) return fail(ctx, RLL_E_INVALID, "more than 2^32 - 1 records");
    if (g->cursor_dirty) {
        e = cudaMemsetAsync(g->cursor, 0, 4 * (size_t)g->H, s);
        if (e != cudaSuccess) return check_cuda(ctx, e, "memset cursors");
        g->cursor_dirty = false;
    }
    void* ws = ws_get(ctx, bucketed_scratch_bytes(n));
    if (!ws) return RLL_E_NOMEM;
    using T = typename Store<P>::T;
    g->cursor_dirty = true;
    e = launch_bucketed_learn<P>(s, g->device, device_sm_count(g->device), rec_key, rec_val, n,
                                 GridDec{g->H * g->M, g->M},
                                 GridRows<P>{(T*)g->Q, (T*)g->C, g->M, g->m, g->p.alpha, g->p.eps}, g->H, g->cursor,
                                 g->touched, g->touched_start, g->touched_len, g->n_touched, g->big, ws,
                                 ctx->d_status, g->M, sp);
    if (e != cudaSuccess) return check_cuda(ctx, e, "learn kernels");
    g->cursor_dirty = false;
    return RLL_OK;
}

// Eq. 1, split-collapse and Eq. 2 of every touched cell in the learning kernels
template <int P>
int learn_split_t(rll_ctx* ctx, rll_grid* g, const rll_tree* t, const uint32_t* rec_key, const float* rec_val,
                  int64_t n)
{
    WithSplit sp;
    sp.cut = g->cut;
    sp.M = g->M;
    sp.nodes = t->nodes;
    sp.parent = t->parent;
    sp.left = t->left;
    sp.right = t->right;
    sp.T = g->p.threshold;
    sp.max_iter = split_steps(g->p);
    sp.n_nodes = 2 * t->n - 1;
    return learn_t<P>(ctx, g, rec_key, rec_val, n, sp);
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

int learn_update_split(rll_ctx* ctx, rll_grid* g, const rll_tree* t, const uint32_t* rec_key, const float* rec_val,
                       int64_t n)
{
    switch (g->p.precision) {
    case RLL_PREC_FP16: return learn_split_t<RLL_PREC_FP16>(ctx, g, t, rec_key, rec_val, n);
    case RLL_PREC_BF16: return learn_split_t<RLL_PREC_BF16>(ctx, g, t, rec_key, rec_val, n);
    default: return learn_split_t<RLL_PREC_FP32>(ctx, g, t, rec_key, rec_val, n);
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
    cudaError_t e = cudaMemsetAsync(g->n_touched, 0, 8 * sizeof(uint32_t), s);
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
