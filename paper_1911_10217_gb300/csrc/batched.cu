// Many uneven scenes (items) in one persistent launch per stage.
//
// Every item is a (grid, tree, G-buffer) triple of its own, with its own
// light count, point count, cut size and Philox seed. One pass:
//   1. k_sample_batched: a persistent kernel (one resident wave of blocks)
//      takes tiles of `tile_points` consecutive points from a global atomic
//      counter; the tile index maps to (item, first point) through a prefix
//      of per-item tile counts. Per point the same device code as the
//      single-grid kernel runs (sample_core.cuh). Records of all items go to
//      one array with keys ((cell_base_i + slot) << 6) | cluster.
//   2. the bucketed learning step of the single grid (bucket_learn.cuh) over
//      all items' cells: records counted and scattered into one bucket per
//      global cell, then one warp (or block) per touched cell orders its bucket
//      by (cluster, sample) and runs Eq. 1, split-collapse (when the pass
//      splits) and Eq. 2 on the item's rows (item found by binary search over
//      the per-item cell prefix).
//   3. k_advance: every item's frame counter += 1 on the device, so the pass
//      can be recorded once as a CUDA graph and launched repeatedly.
// The tile size and the occupancy target of step 1 come from a measured
// search (rll_batch_tune).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bucket_learn.cuh"
#include "learn_core.cuh"
#include "rll_device.cuh"
#include "rll_internal.h"
#include "sample_core.cuh"

namespace rll {
namespace {

constexpr int kBatchThreads = 256;

struct BatchItemDev {
    SampleArgs s;            // sampling arguments (record pointers offset to the item's range)
    void* Q;
    void* C;
    uint32_t* cut;
    const NodeRec* nodes;
    const int32_t* parent;
    const int32_t* left;
    const int32_t* right;
    int64_t n_nodes;
    float alpha, eps, T;
    uint32_t split_iters;    // split-collapse steps per cell
    uint32_t cell_base;      // first global cell of the item
};

template <int P, int MODE, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
k_sample_batched(const BatchItemDev* __restrict__ items, int n_items, const uint32_t* __restrict__ tile_prefix,
                 uint32_t total_tiles, uint32_t tile_points, uint32_t* __restrict__ work)
{
    extern __shared__ float4 s_box[];
    __shared__ uint32_t s_tile;
    __shared__ int s_item;
    __shared__ SampleArgs s_args;  // the current item's arguments
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(work, 1u);
            s_tile = t;
            if (t < total_tiles) {
                int lo = 0, hi = n_items - 1;  // last item whose first tile is <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (tile_prefix[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                s_item = lo;
            }
        }
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= total_tiles) break;
        const int it = s_item;
        if (it != cur) {
            static_assert(sizeof(SampleArgs) % 4 == 0, "SampleArgs is copied as words");
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&items[it].s);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&s_args);
            for (int i = threadIdx.x; i < (int)(sizeof(SampleArgs) / 4); i += blockDim.x) dst[i] = src[i];
            if (items[it].s.boxes_sorted) stage_sorted_boxes(s_box, items[it].s.boxes_sorted, items[it].s.n_boxes);
            else stage_boxes(s_box, items[it].s.boxes, items[it].s.n_boxes);
            cur = it;
        }
        __syncthreads();
        const SampleArgs& a = s_args;
        const int64_t first = (int64_t)(t - tile_prefix[it]) * tile_points;
        const int64_t last = min(first + (int64_t)tile_points, a.n_points);
        for (int64_t p = first + threadIdx.x; p < last; p += blockDim.x) sample_point<P, MODE, false>(a, p, s_box);
        __syncthreads();
    }
}

// Every item's boxes sorted for the shadow test (sort_boxes_block), one block per item, into the
// batch's buffer that the item's descriptor points to.
__global__ void __launch_bounds__(256) k_sort_item_boxes(const BatchItemDev* __restrict__ items, int n_items)
{
    const int it = blockIdx.x;
    if (it >= n_items) return;
    const SampleArgs& a = items[it].s;
    if (a.n_boxes > 0 && a.boxes_sorted)
        sort_boxes_block(a.boxes, a.n_boxes, const_cast<float4*>(a.boxes_sorted));
}

__device__ __forceinline__ int item_of_cell(const uint32_t* __restrict__ cell_prefix, int n_items, uint32_t cell)
{
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cell_prefix[mid] <= cell) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// record key ((cell_base + slot) << kBatchClusterBits) | cluster of many grids
struct BatchDec {
    uint32_t clamp;  // total cells << kBatchClusterBits
    __device__ __forceinline__ bool valid(uint32_t k) const { return k < clamp; }
    __device__ __forceinline__ uint32_t cell(uint32_t k) const { return k >> kBatchClusterBits; }
    __device__ __forceinline__ uint32_t cluster(uint32_t k) const { return k & ((1u << kBatchClusterBits) - 1u); }
};

// rows of a global cell: its item's table row and learning parameters
template <int P>
struct BatchRows {
    const BatchItemDev* items;
    int n_items;
    const uint32_t* cell_prefix;
    __device__ __forceinline__ RowRef<P> row(uint32_t cell) const
    {
        const BatchItemDev& it = items[item_of_cell(cell_prefix, n_items, cell)];
        const int64_t r = (int64_t)(cell - it.cell_base) * it.s.M;
        return RowRef<P>{(typename Store<P>::T*)it.Q + r, (typename Store<P>::T*)it.C + r, it.s.M, it.s.m, it.alpha,
                         it.eps};
    }
};

// split-collapse of a global cell, fused into the learning kernels: its
// item's cut row, light tree, threshold and step limit
struct BatchSplit {
    static constexpr bool kOn = true;
    const BatchItemDev* items;
    int n_items;
    const uint32_t* cell_prefix;
    __device__ __forceinline__ SplitRow row(uint32_t cell) const
    {
        const BatchItemDev& it = items[item_of_cell(cell_prefix, n_items, cell)];
        return SplitRow{it.cut + (int64_t)(cell - it.cell_base) * it.s.M, it.nodes, it.parent, it.left, it.right, it.T,
                        it.split_iters, it.n_nodes};
    }
};

__global__ void k_advance(BatchItemDev* items, int n_items)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_items) items[i].s.frame += 1u;
}

}  // namespace
}  // namespace rll

using namespace rll;

struct rll_batch {
    int device = 0;
    int n = 0;
    uint32_t precision = 0, mode = 0;
    std::vector<BatchItemDev> host;
    BatchItemDev* d_items = nullptr;
    std::vector<uint32_t> points_per_item;
    uint32_t* d_tile_prefix = nullptr;
    uint32_t* d_cell_prefix = nullptr;
    uint32_t* d_work = nullptr;
    uint32_t total_tiles = 0;
    uint32_t tile_points = 1024;
    int min_blocks = 4;
    uint32_t total_cells = 0;
    int64_t n_records = 0;
    uint32_t* rec_key = nullptr;
    float* rec_val = nullptr;
    void* learn_ws = nullptr;          // bucketed_scratch_bytes(cap_records)
    uint32_t* cursor = nullptr;        // [cap_cells] per-cell record cursors, zero between passes
    uint32_t* touched = nullptr;       // [cap_cells]
    uint32_t* touched_start = nullptr; // [cap_cells]
    uint32_t* touched_len = nullptr;   // [cap_cells]
    uint32_t* lists = nullptr;         // [2 cap_cells] cells for the block paths
    uint32_t* n_touched = nullptr;     // [8] learning counters
    int max_boxes = 0;
    uint32_t* status = nullptr;
    float4* box_sorted = nullptr;      // [cap_items][2 kMaxBoxes] every item's boxes sorted by min.x
    int32_t cap_items = 0;
    int64_t cap_records = 0;
    int64_t cap_cells = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    // page-locked staging of the descriptor, cell-prefix and tile-prefix uploads, so that
    // rll_batch_set_items enqueues them without waiting; `staged` is recorded after the
    // last upload from it and waited on before the staging is written again
    void* stage = nullptr;
    BatchItemDev* stage_items = nullptr;   // [cap_items]
    uint32_t* stage_cells = nullptr;       // [cap_items + 1]
    uint32_t* stage_tiles = nullptr;       // [cap_items + 1]
    cudaEvent_t staged = nullptr;
    bool stage_pending = false;
};

namespace {

void free_batch(rll_batch* b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_items);
    cudaFree(b->d_tile_prefix);
    cudaFree(b->d_cell_prefix);
    cudaFree(b->d_work);
    cudaFree(b->rec_key);
    cudaFree(b->rec_val);
    cudaFree(b->learn_ws);
    cudaFree(b->cursor);
    cudaFree(b->touched);
    cudaFree(b->touched_start);
    cudaFree(b->touched_len);
    cudaFree(b->lists);
    cudaFree(b->n_touched);
    cudaFree(b->box_sorted);
    if (b->staged) {
        if (b->stage_pending) cudaEventSynchronize(b->staged);
        cudaEventDestroy(b->staged);
    }
    cudaFreeHost(b->stage);
    delete b;
}

// tiles of every item for a tile size, as an exclusive prefix (n + 1 entries)
std::vector<uint32_t> tile_prefix(const rll_batch* b, uint32_t tile_points)
{
    std::vector<uint32_t> pre(b->n + 1, 0);
    for (int i = 0; i < b->n; ++i)
        pre[i + 1] = pre[i] + (uint32_t)((b->points_per_item[i] + tile_points - 1) / tile_points);
    return pre;
}

// The staging may be written once the uploads enqueued from it have run.
cudaError_t stage_wait(rll_batch* b)
{
    if (!b->stage_pending) return cudaSuccess;
    b->stage_pending = false;
    return cudaEventSynchronize(b->staged);
}

// Uploads the tile prefix through the staging (the caller has waited for it
// and records `staged` afterwards).
int set_tiles_staged(rll_ctx* ctx, rll_batch* b, uint32_t tile_points)
{
    const std::vector<uint32_t> pre = tile_prefix(b, tile_points);
    std::copy(pre.begin(), pre.end(), b->stage_tiles);
    const cudaError_t e = cudaMemcpyAsync(b->d_tile_prefix, b->stage_tiles, sizeof(uint32_t) * (b->n + 1),
                                          cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return check_cuda(ctx, e, "batch tiles");
    b->tile_points = tile_points;
    b->total_tiles = pre[b->n];
    return RLL_OK;
}

int set_tiles(rll_ctx* ctx, rll_batch* b, uint32_t tile_points)
{
    cudaError_t e = stage_wait(b);
    if (e != cudaSuccess) return check_cuda(ctx, e, "batch staging");
    const int rc = set_tiles_staged(ctx, b, tile_points);
    if (rc != RLL_OK) return rc;
    e = cudaEventRecord(b->staged, ctx->stream);
    if (e != cudaSuccess) return check_cuda(ctx, e, "batch staging");
    b->stage_pending = true;
    return RLL_OK;
}

template <int P, int MODE, int MINB>
cudaError_t launch_sample_t(rll_batch* b, cudaStream_t s)
{
    int per_sm = 0;
    const size_t smem = sizeof(float4) * 2 * (size_t)std::max(b->max_boxes, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_batched<P, MODE, MINB>, kBatchThreads, smem);
    const int blocks = std::max(1, per_sm) * device_sm_count(b->device);
    cudaError_t e = cudaMemsetAsync(b->d_work, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_sort_item_boxes<<<b->n, 256, 0, s>>>(b->d_items, b->n);
    k_sample_batched<P, MODE, MINB><<<blocks, kBatchThreads, smem, s>>>(b->d_items, b->n, b->d_tile_prefix,
                                                                        b->total_tiles, b->tile_points, b->d_work);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_sample_p(rll_batch* b, cudaStream_t s)
{
    if (b->mode == RLL_MODE_UNIFORM)
        return b->min_blocks >= 4 ? launch_sample_t<P, RLL_MODE_UNIFORM, 4>(b, s)
                                  : launch_sample_t<P, RLL_MODE_UNIFORM, 3>(b, s);
    if (b->mode == RLL_MODE_DESCENT2)
        return b->min_blocks >= 4 ? launch_sample_t<P, RLL_MODE_DESCENT2, 4>(b, s)
                                  : launch_sample_t<P, RLL_MODE_DESCENT2, 3>(b, s);
    return b->min_blocks >= 4 ? launch_sample_t<P, RLL_MODE_DESCENT, 4>(b, s)
                              : launch_sample_t<P, RLL_MODE_DESCENT, 3>(b, s);
}

cudaError_t launch_sample(rll_batch* b, cudaStream_t s)
{
    switch (b->precision) {
    case RLL_PREC_FP16: return launch_sample_p<RLL_PREC_FP16>(b, s);
    case RLL_PREC_BF16: return launch_sample_p<RLL_PREC_BF16>(b, s);
    default: return launch_sample_p<RLL_PREC_FP32>(b, s);
    }
}

template <int P>
cudaError_t launch_learn_t(rll_batch* b, cudaStream_t s, bool do_split)
{
    cudaError_t e = cudaMemsetAsync(b->n_touched, 0, 8 * sizeof(uint32_t), s);
    if (e != cudaSuccess || b->n_records == 0) return e;
    const int sms = device_sm_count(b->device);
    const BatchDec dec{b->total_cells << kBatchClusterBits};
    const BatchRows<P> rows{b->d_items, b->n, b->d_cell_prefix};
    if (do_split)  // split-collapse fused into the learning kernels
        return launch_bucketed_learn<P>(s, b->device, sms, b->rec_key, b->rec_val, b->n_records, dec, rows,
                                        b->total_cells, b->cursor, b->touched, b->touched_start, b->touched_len,
                                        b->n_touched, b->lists, b->learn_ws, b->status, 1u << kBatchClusterBits,
                                        BatchSplit{b->d_items, b->n, b->d_cell_prefix});
    return launch_bucketed_learn<P>(s, b->device, sms, b->rec_key, b->rec_val, b->n_records, dec, rows,
                                    b->total_cells, b->cursor, b->touched, b->touched_start, b->touched_len,
                                    b->n_touched, b->lists, b->learn_ws, b->status, 1u << kBatchClusterBits);
}

cudaError_t enqueue_pass(rll_batch* b, cudaStream_t s, bool do_split)
{
    cudaError_t e = launch_sample(b, s);
    if (e != cudaSuccess) return e;
    switch (b->precision) {
    case RLL_PREC_FP16: e = launch_learn_t<RLL_PREC_FP16>(b, s, do_split); break;
    case RLL_PREC_BF16: e = launch_learn_t<RLL_PREC_BF16>(b, s, do_split); break;
    default: e = launch_learn_t<RLL_PREC_FP32>(b, s, do_split);
    }
    if (e != cudaSuccess) return e;
    k_advance<<<(b->n + 255) / 256, 256, 0, s>>>(b->d_items, b->n);
    return cudaGetLastError();
}


}  // namespace

extern "C" {

int rll_batch_reserve(rll_ctx* ctx, int32_t max_items, int64_t max_records, int64_t max_cells, rll_batch** out)
{
    if (!ctx || !out) return RLL_E_INVALID;
    *out = nullptr;
    if (max_items < 1 || max_items > 65536) return fail(ctx, RLL_E_INVALID, "max_items must be in [1, 65536]");
    if (max_records < 0 || max_records >= 0xFFFFFFFFll) return fail(ctx, RLL_E_INVALID, "max_records must be < 2^32");
    if (max_cells < 1 || (max_cells << kBatchClusterBits) >= 0xFFFFFFFFll)
        return fail(ctx, RLL_E_INVALID, "max_cells must be in [1, 2^26)");
    DeviceGuard dg(ctx->device);
    rll_batch* b = new (std::nothrow) rll_batch();
    if (!b) return fail(ctx, RLL_E_NOMEM, "host allocation");
    b->device = ctx->device;
    b->status = ctx->d_status;
    b->cap_items = max_items;
    b->cap_records = max_records;
    b->cap_cells = max_cells;
    cudaError_t e = cudaMalloc((void**)&b->rec_key, 4 * std::max<size_t>(max_records, 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->rec_val, 4 * std::max<size_t>(max_records, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->learn_ws, bucketed_scratch_bytes(std::max<int64_t>(max_records, 1)));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->cursor, 4 * (size_t)max_cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->touched, 4 * (size_t)max_cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->touched_start, 4 * (size_t)max_cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->touched_len, 4 * (size_t)max_cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->lists, 8 * (size_t)max_cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->n_touched, 8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->box_sorted, sizeof(float4) * 2 * kMaxBoxes * (size_t)max_items);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->cursor, 0, 4 * (size_t)max_cells, ctx->stream);
    // the learning step's shared-memory opt-in, now rather than during a graph capture
    if (e == cudaSuccess) e = big_smem_attribute<RLL_PREC_FP32, BatchRows<RLL_PREC_FP32>, NoSplit>(ctx->device);
    if (e == cudaSuccess) e = big_smem_attribute<RLL_PREC_FP32, BatchRows<RLL_PREC_FP32>, BatchSplit>(ctx->device);
    if (e == cudaSuccess) e = big_smem_attribute<RLL_PREC_FP16, BatchRows<RLL_PREC_FP16>, NoSplit>(ctx->device);
    if (e == cudaSuccess) e = big_smem_attribute<RLL_PREC_FP16, BatchRows<RLL_PREC_FP16>, BatchSplit>(ctx->device);
    if (e == cudaSuccess) e = big_smem_attribute<RLL_PREC_BF16, BatchRows<RLL_PREC_BF16>, NoSplit>(ctx->device);
    if (e == cudaSuccess) e = big_smem_attribute<RLL_PREC_BF16, BatchRows<RLL_PREC_BF16>, BatchSplit>(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_work, 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_items, sizeof(BatchItemDev) * max_items);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tile_prefix, 4 * (max_items + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_cell_prefix, 4 * (max_items + 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->n_touched, 0, 8 * sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess) {
        const size_t items_b = (sizeof(BatchItemDev) * max_items + 255) & ~(size_t)255;
        const size_t pre_b = (4 * ((size_t)max_items + 1) + 255) & ~(size_t)255;
        e = cudaHostAlloc(&b->stage, items_b + 2 * pre_b, cudaHostAllocDefault);
        if (e == cudaSuccess) {
            b->stage_items = static_cast<BatchItemDev*>(b->stage);
            b->stage_cells = reinterpret_cast<uint32_t*>(static_cast<char*>(b->stage) + items_b);
            b->stage_tiles = reinterpret_cast<uint32_t*>(static_cast<char*>(b->stage) + items_b + pre_b);
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        const int rc = check_cuda(ctx, e, "batch allocation");
        free_batch(b);
        return rc;
    }
    *out = b;
    return RLL_OK;
}

int rll_batch_set_items(rll_ctx* ctx, rll_batch* b, const rll_batch_item* items, int32_t n_items)
{
    if (!ctx || !b) return RLL_E_INVALID;
    if (!items || n_items < 1 || n_items > b->cap_items) return fail(ctx, RLL_E_INVALID, "need 1..max_items items");
    DeviceGuard dg(ctx->device);
    uint32_t precision = 0, mode = 0;
    uint64_t cells = 0, recs = 0;
    int max_boxes = 0;
    for (int i = 0; i < n_items; ++i) {
        const rll_batch_item& it = items[i];
        if (!it.grid || !it.tree) return fail(ctx, RLL_E_INVALID, "item without grid or tree");
        const rll_grid* g = it.grid;
        if (g->n_lights != it.tree->n) return fail(ctx, RLL_E_INVALID, "item grid built for another tree");
        if (i == 0) {
            precision = g->p.precision;
            mode = g->p.in_cluster_mode;
        } else if (g->p.precision != precision || g->p.in_cluster_mode != mode) {
            return fail(ctx, RLL_E_INVALID, "all items need the same table precision and in-cluster mode");
        }
        if (g->M > (1u << kBatchClusterBits)) return fail(ctx, RLL_E_INVALID, "batched cut size must be <= 64");
        for (int j = 0; j < i; ++j)
            if (items[j].grid == g) return fail(ctx, RLL_E_INVALID, "a grid appears twice in one batch");
        if (it.n_points < 0 || it.n_points > 0xFFFFFFFFll || it.spp < 1 || it.spp > 65536 ||
            (uint64_t)it.n_points * it.spp >= 0xFFFFFFFFull)
            return fail(ctx, RLL_E_INVALID, "bad n_points / spp");
        if (it.n_boxes < 0 || it.n_boxes > kMaxBoxes || (it.n_boxes > 0 && !it.boxes))
            return fail(ctx, RLL_E_INVALID, "bad boxes");
        if (it.n_points > 0 && (!it.pos || !it.nrm || !it.albedo || !it.rgb))
            return fail(ctx, RLL_E_INVALID, "NULL G-buffer or rgb");
        cells += g->H;
        recs += (uint64_t)it.n_points * it.spp;
        max_boxes = std::max(max_boxes, (int)it.n_boxes);
    }
    if ((int64_t)cells > b->cap_cells) return fail(ctx, RLL_E_INVALID, "items exceed the batch's cell capacity");
    if ((int64_t)recs > b->cap_records) return fail(ctx, RLL_E_INVALID, "items exceed the batch's record capacity");
    if (b->graph) {  // a recorded pass holds the old sizes
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->n = n_items;
    b->precision = precision;
    b->mode = mode;
    b->max_boxes = max_boxes;
    b->total_cells = (uint32_t)cells;
    b->n_records = (int64_t)recs;
    b->host.resize(n_items);
    b->points_per_item.resize(n_items);
    std::vector<uint32_t> cell_pre(n_items + 1, 0);
    uint64_t rec_off = 0;
    for (int i = 0; i < n_items; ++i) {
        const rll_batch_item& it = items[i];
        rll_grid* g = it.grid;
        const rll_tree* t = it.tree;
        BatchItemDev& d = b->host[i];
        SampleArgs& a = d.s;
        a = SampleArgs{};
        a.pos = it.pos;
        a.nrm = it.nrm;
        a.albedo = it.albedo;
        a.n_points = it.n_points;
        a.boxes = it.boxes;
        a.n_boxes = it.n_boxes;
        a.boxes_sorted = it.n_boxes > 0 ? b->box_sorted + 2 * kMaxBoxes * (size_t)i : nullptr;
        a.keys = g->keys;
        a.cut = g->cut;
        a.C = g->C;
        a.Hl = g->Hl;
        a.levels = g->levels;
        a.footprint = nullptr;
        a.M = g->M;
        a.m = g->m;
        a.def_cut = g->def_cut;
        a.def_C = g->def_C;
        for (int k = 0; k < 3; ++k) a.origin[k] = g->p.origin[k];
        a.h = g->p.cell_size;
        a.nb = g->p.normal_bins;
        a.jitter = g->p.jitter;
        a.reward_mode = g->p.reward_mode;
        a.pairs = t->pairs;
        a.quads = t->quads;
        a.nodes = t->nodes;
        a.lights = t->lights;
        a.light_cdf = t->light_cdf;
        a.n_lights = t->n;
        a.seed = it.seed;
        a.frame = it.frame;
        a.spp = it.spp;
        a.rgb = it.rgb;
        a.rec_key = b->rec_key + rec_off;
        a.rec_val = b->rec_val + rec_off;
        a.status = b->status;
        a.key_cells = 1;
        a.cell_base = cell_pre[i];
        d.Q = g->Q;
        d.C = g->C;
        d.cut = g->cut;
        d.nodes = t->nodes;
        d.parent = t->parent;
        d.left = t->left;
        d.right = t->right;
        d.n_nodes = 2 * t->n - 1;
        d.alpha = g->p.alpha;
        d.eps = g->p.eps;
        d.T = g->p.threshold;
        d.split_iters = split_steps(g->p);
        d.cell_base = cell_pre[i];
        cell_pre[i + 1] = cell_pre[i] + g->H;
        rec_off += (uint64_t)it.n_points * it.spp;
        b->points_per_item[i] = (uint32_t)it.n_points;
    }
    // through the page-locked staging: the copies are enqueued without waiting (only a previous
    // upload from the staging that has not run yet is waited for)
    cudaError_t e = stage_wait(b);
    if (e == cudaSuccess) {
        std::copy(b->host.begin(), b->host.end(), b->stage_items);
        std::copy(cell_pre.begin(), cell_pre.end(), b->stage_cells);
        e = cudaMemcpyAsync(b->d_items, b->stage_items, sizeof(BatchItemDev) * n_items, cudaMemcpyHostToDevice,
                            ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_cell_prefix, b->stage_cells, 4 * (n_items + 1), cudaMemcpyHostToDevice,
                            ctx->stream);
    int rc = check_cuda(ctx, e, "batch upload");
    if (rc == RLL_OK) rc = set_tiles_staged(ctx, b, b->tile_points);
    if (rc == RLL_OK) {
        e = cudaEventRecord(b->staged, ctx->stream);
        if (e == cudaSuccess) b->stage_pending = true;
        rc = check_cuda(ctx, e, "batch staging");
    }
    return rc;
}

int rll_batch_create(rll_ctx* ctx, const rll_batch_item* items, int32_t n_items, rll_batch** out)
{
    if (!ctx || !out) return RLL_E_INVALID;
    *out = nullptr;
    if (!items || n_items < 1) return fail(ctx, RLL_E_INVALID, "need at least one item");
    int64_t recs = 0, cells = 0;
    for (int i = 0; i < n_items; ++i) {
        if (!items[i].grid) return fail(ctx, RLL_E_INVALID, "item without grid");
        recs += std::max<int64_t>(items[i].n_points, 0) * std::max(items[i].spp, 1);
        cells += items[i].grid->H;
    }
    rll_batch* b = nullptr;
    int rc = rll_batch_reserve(ctx, n_items, recs, cells, &b);
    if (rc != RLL_OK) return rc;
    rc = rll_batch_set_items(ctx, b, items, n_items);
    if (rc != RLL_OK) {
        rll_batch_destroy(b);
        return rc;
    }
    *out = b;
    return RLL_OK;
}

int rll_batch_set_config(rll_ctx* ctx, rll_batch* b, int32_t tile_points, int32_t min_blocks)
{
    if (!ctx || !b) return RLL_E_INVALID;
    if (tile_points < 32 || tile_points > (1 << 20)) return fail(ctx, RLL_E_INVALID, "tile_points must be in [32, 2^20]");
    if (min_blocks != 3 && min_blocks != 4) return fail(ctx, RLL_E_INVALID, "min_blocks must be 3 or 4");
    DeviceGuard dg(ctx->device);
    b->min_blocks = min_blocks;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    const int rc = set_tiles(ctx, b, (uint32_t)tile_points);
    return rc == RLL_OK ? check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "batch config") : rc;
}

int rll_batch_tune(rll_ctx* ctx, rll_batch* b, int32_t* tile_points_out, int32_t* min_blocks_out)
{
    if (!ctx || !b) return RLL_E_INVALID;
    DeviceGuard dg(ctx->device);
    const uint32_t tiles[] = {128, 256, 512, 1024, 2048, 4096, 8192};
    const int minbs[] = {3, 4};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return check_cuda(ctx, cudaGetLastError(), "tune events");
    float best = 1e30f;
    uint32_t best_tile = b->tile_points;
    int best_mb = b->min_blocks;
    int rc = RLL_OK;
    for (int mb : minbs) {
        for (uint32_t tp : tiles) {
            b->min_blocks = mb;
            rc = set_tiles(ctx, b, tp);
            if (rc != RLL_OK) break;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {  // first repetition warms the caches and the hash tables
                cudaEventRecord(e0, ctx->stream);
                cudaError_t e = launch_sample(b, ctx->stream);
                cudaEventRecord(e1, ctx->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    rc = check_cuda(ctx, e, "tune");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_min = std::min(ms_min, ms);
            }
            if (rc != RLL_OK) break;
            if (ms_min < best) {
                best = ms_min;
                best_tile = tp;
                best_mb = mb;
            }
        }
        if (rc != RLL_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RLL_OK) return rc;
    if (tile_points_out) *tile_points_out = (int32_t)best_tile;
    if (min_blocks_out) *min_blocks_out = best_mb;
    return rll_batch_set_config(ctx, b, (int32_t)best_tile, best_mb);
}

int rll_batch_run(rll_ctx* ctx, rll_batch* b, int32_t do_split)
{
    if (!ctx || !b) return RLL_E_INVALID;
    DeviceGuard dg(ctx->device);
    return check_cuda(ctx, enqueue_pass(b, ctx->stream, do_split != 0), "batch pass");
}

int rll_batch_capture(rll_ctx* ctx, rll_batch* b, int32_t do_split)
{
    if (!ctx || !b) return RLL_E_INVALID;
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaSuccess;
    if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return check_cuda(ctx, e, "capture stream");
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    // the pass reads state written by earlier work on the context stream
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return check_cuda(ctx, e, "capture");
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return check_cuda(ctx, e, "begin capture");
    const cudaError_t pe = enqueue_pass(b, b->cap_stream, do_split != 0);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (pe != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return check_cuda(ctx, pe, "capture pass");
    }
    if (e != cudaSuccess) return check_cuda(ctx, e, "end capture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    return check_cuda(ctx, e, "instantiate graph");
}

int rll_batch_launch(rll_ctx* ctx, rll_batch* b)
{
    if (!ctx || !b) return RLL_E_INVALID;
    if (!b->graph) return fail(ctx, RLL_E_INVALID, "no recorded pass: call rll_batch_capture first");
    DeviceGuard dg(ctx->device);
    return check_cuda(ctx, cudaGraphLaunch(b->graph, ctx->stream), "graph launch");
}

int rll_batch_destroy(rll_batch* b)
{
    if (!b) return RLL_OK;
    DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    free_batch(b);
    return RLL_OK;
}

}  // extern "C"
