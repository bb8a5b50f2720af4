// Render-time sampling (Section 3, "Main contribution"; Section 3.1: "sampling
// the cdf is performed by a standard binary search").
//
// One thread per shading point (spp samples in a loop); occluder boxes staged
// in shared memory once per block. Per sample:
//   hash lookup / lazy insert of the (jittered) 5-d cell   (64-bit CAS)
//   binary search of the cell's C for the cluster s        (log2 m loads of one row)
//   in-cluster choice: bound-driven descent (one 80-byte record of both
//   children per level, both bounds in packed f32x2 arithmetic) or a uniform
//   pick over the cluster's lights
//   uniform point on the light triangle, contribution, shadow segment vs the
//   boxes (sorted by min.x once per call; only the run that can meet the
//   segment is tested)
//   estimate accumulation and one learning record (key, |c|).
// The decisions (cell, branch, visibility) are exact binary32 formulas; the
// cdf and descent comparisons u * total < c are made exactly with one fma.

#include <cuda_runtime.h>

#include "rll_device.cuh"
#include "rll_internal.h"
#include "sample_core.cuh"

namespace rll {
namespace {

constexpr int kThreads = 256;

// THREADS x MINB: block size and the resident blocks per SM the registers are
// held to (128 x 8: 64 registers, 32 warps per SM; 128 x 6: 80 registers).
// Blocks of 128 rather than 256 threads at the same occupancy: a block's
// slowest descent holds fewer lanes back (measured 1 % faster; 64-thread
// blocks lose it again to staging the boxes twice as often).
template <int P, int MODE, bool DBG, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_sample(SampleArgs a)
{
    pdl_begin();
    extern __shared__ float4 s_box[];
    if (a.boxes_sorted) stage_sorted_boxes(s_box, a.boxes_sorted, a.n_boxes);
    else stage_boxes(s_box, a.boxes, a.n_boxes);
    __syncthreads();
    const int64_t p = a.p_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.p_end) return;
    sample_point<P, MODE, DBG>(a, p, s_box);
}

// Energy-based baseline (Section 4): inversion of the cdf of leaf power.
__global__ void __launch_bounds__(kThreads) k_sample_power(SampleArgs a, int32_t* light_out)
{
    extern __shared__ float4 s_box[];
    stage_boxes(s_box, a.boxes, a.n_boxes);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_points) return;
    const int64_t np = a.n_points;
    const float x0 = a.pos[p], x1 = a.pos[np + p], x2 = a.pos[2 * np + p];
    const float n0 = a.nrm[p], n1 = a.nrm[np + p], n2 = a.nrm[2 * np + p];
    const float alb = a.albedo[p];
    const int64_t nl = a.n_lights;
    const float total = a.light_cdf[nl - 1];
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;
    for (int j = 0; j < a.spp; ++j) {
        const uint32_t sid = (uint32_t)(p * a.spp + j);
        SampleStream rs;
        rs.init(a.seed, sid, a.frame);
        const float u = rs.draw(kDrawCut);
        int64_t lo = 0, hi = nl - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (__fmaf_rn(-u, total, a.light_cdf[mid]) > 0.0f) hi = mid;
            else lo = mid + 1;
        }
        const float pl = a.nodes[nl - 1 + lo].phi / total;
        const LightRec Lr = load_light(a.lights + lo);
        const ShadeOut o = shade(Lr, x0, x1, x2, n0, n1, n2, alb, pl, 1.0f, rs.draw(kDrawTriA), rs.draw(kDrawTriB),
                                 s_box, a.n_boxes, 0);
        acc0 += o.est[0];
        acc1 += o.est[1];
        acc2 += o.est[2];
        if (light_out) light_out[sid] = (int32_t)lo;
    }
    const float inv_spp = 1.0f / (float)a.spp;
    a.rgb[p] = acc0 * inv_spp;
    a.rgb[np + p] = acc1 * inv_spp;
    a.rgb[2 * np + p] = acc2 * inv_spp;
}

// The occluder boxes sorted for the shadow test (sort_boxes_block in sample_core.cuh), one block.
constexpr int kSortBoxThreads = 256;

__global__ void __launch_bounds__(kSortBoxThreads) k_sort_boxes(const float* __restrict__ boxes, int n,
                                                                float4* __restrict__ out)
{
    pdl_begin();
    sort_boxes_block(boxes, n, out);
}

template <int P, int MODE, bool DBG, int THREADS, int MINB>
cudaError_t launch(const SampleArgs& a, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((a.p_end - a.p_begin + THREADS - 1) / THREADS);
    const size_t smem = sizeof(float4) * 2 * (size_t)a.n_boxes;
    return launch_pdl(k_sample<P, MODE, DBG, THREADS, MINB>, dim3(blocks), dim3(THREADS), smem, s, a);
}

template <int P, int MODE>
cudaError_t launch_m(const SampleArgs& a, bool dbg, int minb, cudaStream_t s)
{
    if (dbg) return launch<P, MODE, true, 256, 3>(a, s);
    return minb == 4 ? launch<P, MODE, false, 128, 8>(a, s) : launch<P, MODE, false, 128, 6>(a, s);
}

template <int P>
cudaError_t launch_p(const SampleArgs& a, int mode, bool dbg, int minb, cudaStream_t s)
{
    if (mode == RLL_MODE_UNIFORM) return launch_m<P, RLL_MODE_UNIFORM>(a, dbg, minb, s);
    if (mode == RLL_MODE_DESCENT2) return launch_m<P, RLL_MODE_DESCENT2>(a, dbg, minb, s);
    return launch_m<P, RLL_MODE_DESCENT>(a, dbg, minb, s);
}

}  // namespace

int sample_and_shade(rll_ctx* ctx, rll_grid* g, const rll_tree* t, const float* pos, const float* nrm,
                     const float* albedo, const float* footprint, int64_t n_points, const float* boxes, int n_boxes,
                     uint64_t seed,
                     uint32_t frame, int spp, float* rgb, uint32_t* rec_key, float* rec_val,
                     const rll_sample_debug* dbg)
{
    const void* sorted = nullptr;
    const int rc = sort_boxes(ctx, boxes, n_boxes, ctx->stream, &sorted);
    if (rc != RLL_OK) return rc;
    return sample_and_shade_range(ctx, g, t, pos, nrm, albedo, footprint, n_points, 0, n_points, boxes, n_boxes, seed,
                                  frame, spp, rgb, rec_key, rec_val, dbg, ctx->stream, sorted);
}

int sort_boxes(rll_ctx* ctx, const float* boxes, int n_boxes, cudaStream_t stream, const void** out)
{
    *out = nullptr;
    if (n_boxes <= 0) return RLL_OK;
    if (!ctx->box_sorted) {
        if (cudaMalloc(&ctx->box_sorted, sizeof(float4) * 2 * (size_t)kMaxBoxes) != cudaSuccess) {
            cudaGetLastError();
            ctx->box_sorted = nullptr;
            return fail(ctx, RLL_E_NOMEM, "cannot allocate the sorted boxes");
        }
    }
    const int rc = check_cuda(ctx,
                              launch_pdl(k_sort_boxes, dim3(1), dim3(kSortBoxThreads), 0, stream, boxes, n_boxes,
                                         static_cast<float4*>(ctx->box_sorted)),
                              "sort boxes");
    if (rc == RLL_OK) *out = ctx->box_sorted;
    return rc;
}

int sample_and_shade_range(rll_ctx* ctx, rll_grid* g, const rll_tree* t, const float* pos, const float* nrm,
                           const float* albedo, const float* footprint, int64_t n_points, int64_t p_begin,
                           int64_t p_end, const float* boxes, int n_boxes, uint64_t seed, uint32_t frame, int spp,
                           float* rgb, uint32_t* rec_key, float* rec_val, const rll_sample_debug* dbg,
                           cudaStream_t stream, const void* sorted_boxes)
{
    if (p_end <= p_begin) return RLL_OK;
    SampleArgs a{};
    a.boxes_sorted = static_cast<const float4*>(sorted_boxes);
    a.pos = pos;
    a.nrm = nrm;
    a.albedo = albedo;
    a.n_points = n_points;
    a.p_begin = p_begin;
    a.p_end = p_end;
    a.boxes = boxes;
    a.n_boxes = n_boxes;
    a.keys = g->keys;
    a.cut = g->cut;
    a.C = g->C;
    a.Hl = g->Hl;
    a.levels = g->levels;
    a.footprint = footprint;
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
    a.seed = seed;
    a.frame = frame;
    a.spp = spp;
    a.rgb = rgb;
    a.rec_key = rec_key;
    a.rec_val = rec_val;
    a.status = ctx->d_status;
    const bool use_dbg = dbg && (dbg->light || dbg->p_cut || dbg->p_in);
    if (use_dbg) {
        a.dbg_light = dbg->light;
        a.dbg_pcut = dbg->p_cut;
        a.dbg_pin = dbg->p_in;
    }
    cudaError_t e;
    const int minb = ctx->sample_min_blocks;
    const int mode = g->p.in_cluster_mode;
    switch (g->p.precision) {
    case RLL_PREC_FP16: e = launch_p<RLL_PREC_FP16>(a, mode, use_dbg, minb, stream); break;
    case RLL_PREC_BF16: e = launch_p<RLL_PREC_BF16>(a, mode, use_dbg, minb, stream); break;
    default: e = launch_p<RLL_PREC_FP32>(a, mode, use_dbg, minb, stream);
    }
    return check_cuda(ctx, e, "sample_and_shade");
}

int sample_power(rll_ctx* ctx, const rll_tree* t, const float* pos, const float* nrm, const float* albedo,
                 int64_t n_points, const float* boxes, int n_boxes, uint64_t seed, uint32_t frame, int spp,
                 float* rgb, int32_t* light_out)
{
    if (n_points == 0) return RLL_OK;
    SampleArgs a{};
    a.pos = pos;
    a.nrm = nrm;
    a.albedo = albedo;
    a.n_points = n_points;
    a.boxes = boxes;
    a.n_boxes = n_boxes;
    a.nodes = t->nodes;
    a.lights = t->lights;
    a.light_cdf = t->light_cdf;
    a.n_lights = t->n;
    a.seed = seed;
    a.frame = frame;
    a.spp = spp;
    a.rgb = rgb;
    const unsigned blocks = (unsigned)((n_points + kThreads - 1) / kThreads);
    k_sample_power<<<blocks, kThreads, sizeof(float4) * 2 * n_boxes, ctx->stream>>>(a, light_out);
    return check_cuda(ctx, cudaGetLastError(), "sample_power");
}

}  // namespace rll
