// C ABI of the library (include/rll.h): argument checks, handle lifetimes,
// library-owned scratch, host staging. Every entry point returns a status
// and never throws.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "rll_device.cuh"
#include "rll_internal.h"

namespace rll {

int fail(rll_ctx* ctx, int code, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int check_cuda(rll_ctx* ctx, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return RLL_OK;
    if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RLL_E_NOMEM : RLL_E_CUDA;
}

void* ws_get(rll_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return ctx->ws;
    // the old buffer may still be read by enqueued work
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    const size_t want = bytes + bytes / 4 + 4096;
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "cannot allocate " + std::to_string(want) + " bytes of scratch";
        return nullptr;
    }
    ctx->ws_bytes = want;
    return ctx->ws;
}

namespace {

size_t elem_bytes(uint32_t precision) { return precision == RLL_PREC_FP32 ? 4 : 2; }

void free_tree(rll_tree* t)
{
    if (!t) return;
    cudaFree(t->nodes);
    cudaFree(t->pairs);
    cudaFree(t->quads);
    cudaFree(t->lights);
    cudaFree(t->perm);
    cudaFree(t->left);
    cudaFree(t->right);
    cudaFree(t->parent);
    cudaFree(t->light_cdf);
    delete t;
}

void free_grid(rll_grid* g)
{
    if (!g) return;
    cudaFree(g->keys);
    cudaFree(g->cut);
    cudaFree(g->Q);
    cudaFree(g->C);
    cudaFree(g->def_cut);
    cudaFree(g->def_Q);
    cudaFree(g->def_C);
    cudaFree(g->touched);
    cudaFree(g->touched_start);
    cudaFree(g->touched_len);
    cudaFree(g->n_touched);
    cudaFree(g->cursor);
    cudaFree(g->big);
    delete g;
}

int check_params(rll_ctx* ctx, const rll_grid_params* p)
{
    if (!p) return fail(ctx, RLL_E_INVALID, "params is NULL");
    const uint32_t H = p->table_size;
    if (H < 16 || H > (1u << 26) || (H & (H - 1)) != 0)
        return fail(ctx, RLL_E_INVALID, "table_size must be a power of two in [16, 2^26]");
    if (p->cut_size < 1 || p->cut_size > (uint32_t)kMaxCut) return fail(ctx, RLL_E_INVALID, "cut_size must be in [1, 256]");
    if (p->levels > 16) return fail(ctx, RLL_E_INVALID, "levels must be in [0, 16]");
    const uint64_t total = (uint64_t)H * (p->levels ? p->levels : 1u);
    if (total > (1ull << 27)) return fail(ctx, RLL_E_INVALID, "levels * table_size must be <= 2^27");
    if (total * p->cut_size > (1ull << 31))
        return fail(ctx, RLL_E_INVALID, "levels * table_size * cut_size must be <= 2^31");
    if (!(p->cell_size > 0.0f) || !std::isfinite(p->cell_size)) return fail(ctx, RLL_E_INVALID, "cell_size must be > 0");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(p->origin[k])) return fail(ctx, RLL_E_INVALID, "origin must be finite");
    if (p->normal_bins < 1 || p->normal_bins > 255) return fail(ctx, RLL_E_INVALID, "normal_bins must be in [1, 255]");
    if (p->jitter > 1) return fail(ctx, RLL_E_INVALID, "jitter must be 0 or 1");
    if (p->precision > RLL_PREC_BF16) return fail(ctx, RLL_E_INVALID, "unknown precision");
    if (p->in_cluster_mode > RLL_MODE_DESCENT2) return fail(ctx, RLL_E_INVALID, "unknown in_cluster_mode");
    if (p->reward_mode > RLL_REWARD_LITERAL) return fail(ctx, RLL_E_INVALID, "unknown reward_mode");
    if (!(p->alpha >= 0.0f && p->alpha <= 1.0f)) return fail(ctx, RLL_E_INVALID, "alpha must be in [0, 1]");
    if (!(p->threshold > 0.0f) || !std::isfinite(p->threshold)) return fail(ctx, RLL_E_INVALID, "threshold must be > 0");
    if (!(p->eps >= 0.0f) || !std::isfinite(p->eps)) return fail(ctx, RLL_E_INVALID, "eps must be >= 0");
    if (!(p->q_init > 0.0f) || !std::isfinite(p->q_init)) return fail(ctx, RLL_E_INVALID, "q_init must be > 0");
    if (p->split_iterations > kMaxSplitIterations)
        return fail(ctx, RLL_E_INVALID, "split_iterations must be in [0, 256]");
    return RLL_OK;
}

// Breadth-first initial cut of min(M, n) nodes (Section 3), sorted by range
// begin. Topology and node begins are copied to the host once per grid.
int initial_cut(rll_ctx* ctx, const rll_tree* t, uint32_t M, std::vector<uint32_t>* cut)
{
    const int64_t n = t->n;
    const uint32_t m = (uint32_t)std::min<int64_t>(M, n);
    std::vector<int32_t> left(std::max<int64_t>(n - 1, 1)), right(std::max<int64_t>(n - 1, 1));
    std::vector<uint32_t> begin(2 * n - 1);
    cudaError_t e = cudaSuccess;
    if (n > 1) {
        e = cudaMemcpyAsync(left.data(), t->left, sizeof(int32_t) * (n - 1), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(right.data(), t->right, sizeof(int32_t) * (n - 1), cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(begin.data(), sizeof(uint32_t), &t->nodes[0].begin, sizeof(NodeRec), sizeof(uint32_t),
                              (size_t)(2 * n - 1), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return check_cuda(ctx, e, "initial cut: copy tree");
    std::deque<int64_t> q;
    q.push_back(0);
    while (q.size() < m) {
        const int64_t id = q.front();
        q.pop_front();
        if (id >= n - 1) {
            q.push_back(id);
        } else {
            q.push_back(left[id]);
            q.push_back(right[id]);
        }
    }
    cut->assign(q.begin(), q.end());
    std::sort(cut->begin(), cut->end(), [&](uint32_t a, uint32_t b) { return begin[a] < begin[b]; });
    return RLL_OK;
}

}  // namespace
}  // namespace rll

using namespace rll;

extern "C" {

int rll_ctx_create(rll_ctx** out, int device, void* cuda_stream)
{
    if (!out) return RLL_E_INVALID;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return RLL_E_CUDA;
    }
    rll_ctx* ctx = new (std::nothrow) rll_ctx();
    if (!ctx) return RLL_E_NOMEM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    if (cudaMalloc(&ctx->d_status, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return RLL_E_NOMEM;
    }
    *out = ctx;
    return RLL_OK;
}

int rll_ctx_set_stream(rll_ctx* ctx, void* cuda_stream)
{
    if (!ctx) return RLL_E_INVALID;
    ctx->stream = (cudaStream_t)cuda_stream;
    return RLL_OK;
}

int rll_ctx_set_option(rll_ctx* ctx, const char* name, int64_t value)
{
    if (!ctx || !name) return RLL_E_INVALID;
    const std::string n(name);
    if (n == "host_zero_copy") {
        if (value != 0 && value != 1) return fail(ctx, RLL_E_INVALID, "host_zero_copy must be 0 or 1");
        ctx->host_zero_copy = (int)value;
        return RLL_OK;
    }
    if (n == "host_chunks") {
        if (value < 1 || value > RLL_HOST_MAX_CHUNKS)
            return fail(ctx, RLL_E_INVALID, "host_chunks must be in [1, " + std::to_string(RLL_HOST_MAX_CHUNKS) + "]");
        ctx->host_chunks = (int)value;
        return RLL_OK;
    }
    if (n == "sample_min_blocks") {
        if (value != 3 && value != 4) return fail(ctx, RLL_E_INVALID, "sample_min_blocks must be 3 or 4");
        ctx->sample_min_blocks = (int)value;
        return RLL_OK;
    }
    return fail(ctx, RLL_E_INVALID, "unknown option " + n);
}

int rll_ctx_destroy(rll_ctx* ctx)
{
    if (!ctx) return RLL_OK;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_status);
    cudaFree(ctx->ws);
    cudaFree(ctx->stage);
    cudaFree(ctx->box_sorted);
    if (ctx->pipe_ready) {
        cudaStreamSynchronize(ctx->up);
        cudaStreamSynchronize(ctx->down);
        cudaStreamSynchronize(ctx->comp2);
        for (cudaEvent_t ev : ctx->ev) cudaEventDestroy(ev);
        cudaStreamDestroy(ctx->up);
        cudaStreamDestroy(ctx->down);
        cudaStreamDestroy(ctx->comp2);
    }
    delete ctx;
    return RLL_OK;
}

const char* rll_last_error(const rll_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int rll_sync_status(rll_ctx* ctx)
{
    if (!ctx) return -RLL_E_INVALID;
    DeviceGuard g(ctx->device);
    uint32_t bits = 0;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&bits, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        check_cuda(ctx, e, "sync_status");
        return -RLL_E_CUDA;
    }
    return (int)bits;
}

int rll_build_light_tree_ex(rll_ctx* ctx, const float* tri, const float* emission, int64_t n, int32_t builder,
                            rll_tree** out)
{
    if (!ctx || !out) return RLL_E_INVALID;
    *out = nullptr;
    if (!tri || !emission) return fail(ctx, RLL_E_INVALID, "tri / emission is NULL");
    if (n < 1 || n > (1ll << 24)) return fail(ctx, RLL_E_INVALID, "light count must be in [1, 2^24]");
    if (builder != RLL_TREE_LBVH && builder != RLL_TREE_SAOH && builder != RLL_TREE_MEDIAN)
        return fail(ctx, RLL_E_INVALID, "unknown builder");
    DeviceGuard g(ctx->device);
    rll_tree* t = new (std::nothrow) rll_tree();
    if (!t) return fail(ctx, RLL_E_NOMEM, "host allocation");
    t->device = ctx->device;
    const int rc = build_tree(ctx, tri, emission, n, builder, t);
    if (rc != RLL_OK) {
        free_tree(t);
        return rc;
    }
    *out = t;
    return RLL_OK;
}

int rll_build_light_tree(rll_ctx* ctx, const float* tri, const float* emission, int64_t n, rll_tree** out)
{
    return rll_build_light_tree_ex(ctx, tri, emission, n, RLL_TREE_LBVH, out);
}

int rll_tree_update_emission(rll_ctx* ctx, rll_tree* tree, const float* emission)
{
    if (!ctx || !tree || !emission) return ctx ? fail(ctx, RLL_E_INVALID, "NULL argument") : RLL_E_INVALID;
    DeviceGuard g(ctx->device);
    return tree_update_emission(ctx, tree, emission);
}

int64_t rll_tree_num_lights(const rll_tree* tree) { return tree ? tree->n : 0; }

int rll_tree_export(rll_ctx* ctx, const rll_tree* t, uint32_t* perm, int32_t* left, int32_t* right, int32_t* parent,
                    uint32_t* begin, uint32_t* end, float* rec)
{
    if (!ctx || !t) return RLL_E_INVALID;
    DeviceGuard g(ctx->device);
    const int64_t n = t->n, nn = 2 * n - 1;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (perm) e = cudaMemcpyAsync(perm, t->perm, 4 * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && left && n > 1) e = cudaMemcpyAsync(left, t->left, 4 * (n - 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && right && n > 1) e = cudaMemcpyAsync(right, t->right, 4 * (n - 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && parent) e = cudaMemcpyAsync(parent, t->parent, 4 * nn, cudaMemcpyDeviceToHost, s);
    std::vector<NodeRec> nodes;
    if (e == cudaSuccess && (begin || end || rec)) {
        nodes.resize(nn);
        e = cudaMemcpyAsync(nodes.data(), t->nodes, sizeof(NodeRec) * nn, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "tree export");
    for (int64_t i = 0; i < (int64_t)nodes.size(); ++i) {
        const NodeRec& r = nodes[i];
        if (begin) begin[i] = r.begin;
        if (end) end[i] = r.end;
        if (rec) {
            float* o = rec + i * 11;
            for (int k = 0; k < 3; ++k) {
                o[k] = r.bmin[k];
                o[3 + k] = r.bmax[k];
                o[7 + k] = r.axis[k];
            }
            o[6] = r.phi;
            o[10] = r.cos_t;
        }
    }
    return RLL_OK;
}

int rll_tree_destroy(rll_tree* tree)
{
    if (!tree) return RLL_OK;
    DeviceGuard g(tree->device);
    cudaDeviceSynchronize();
    free_tree(tree);
    return RLL_OK;
}

int rll_create_grid(rll_ctx* ctx, const rll_tree* tree, const rll_grid_params* params, rll_grid** out)
{
    if (!ctx || !out) return RLL_E_INVALID;
    *out = nullptr;
    if (!tree) return fail(ctx, RLL_E_INVALID, "tree is NULL");
    int rc = check_params(ctx, params);
    if (rc != RLL_OK) return rc;
    DeviceGuard dg(ctx->device);
    rll_grid* g = new (std::nothrow) rll_grid();
    if (!g) return fail(ctx, RLL_E_NOMEM, "host allocation");
    g->device = ctx->device;
    g->p = *params;
    g->Hl = params->table_size;
    g->levels = params->levels ? params->levels : 1u;
    g->H = g->Hl * g->levels;
    g->M = params->cut_size;
    g->n_lights = tree->n;
    std::vector<uint32_t> cut;
    rc = initial_cut(ctx, tree, g->M, &cut);
    if (rc != RLL_OK) {
        free_grid(g);
        return rc;
    }
    g->m = (uint32_t)cut.size();
    const size_t eb = elem_bytes(params->precision);
    const size_t rows = (size_t)g->H * g->M;
    cudaError_t e = cudaMalloc((void**)&g->keys, 8 * (size_t)g->H);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->cut, 4 * rows);
    if (e == cudaSuccess) e = cudaMalloc(&g->Q, eb * rows);
    if (e == cudaSuccess) e = cudaMalloc(&g->C, eb * rows);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->def_cut, 4 * g->m);
    if (e == cudaSuccess) e = cudaMalloc(&g->def_Q, eb * g->m);
    if (e == cudaSuccess) e = cudaMalloc(&g->def_C, eb * g->m);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->touched, 4 * (size_t)g->H);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->touched_start, 4 * (size_t)g->H);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->touched_len, 4 * (size_t)g->H);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->n_touched, 8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->cursor, 4 * (size_t)g->H);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->big, 8 * (size_t)g->H);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->keys, 0xFF, 8 * (size_t)g->H, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->n_touched, 0, 8 * sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->cursor, 0, 4 * (size_t)g->H, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->def_cut, cut.data(), 4 * g->m, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        rc = check_cuda(ctx, e, "create_grid");
        free_grid(g);
        return rc;
    }
    rc = grid_init(ctx, g);
    if (rc == RLL_OK) rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "create_grid");
    if (rc != RLL_OK) {
        free_grid(g);
        return rc;
    }
    *out = g;
    return RLL_OK;
}

uint32_t rll_grid_cut_len(const rll_grid* grid) { return grid ? grid->m : 0; }

int rll_grid_touched_cells(rll_ctx* ctx, const rll_grid* g, int64_t* out)
{
    if (!ctx) return RLL_E_INVALID;
    if (!g || !out) return fail(ctx, RLL_E_INVALID, "grid / out is NULL");
    DeviceGuard dg(ctx->device);
    uint32_t n = 0;
    cudaError_t e = cudaMemcpyAsync(&n, g->n_touched, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return check_cuda(ctx, e, "grid touched cells");
    *out = (int64_t)n;
    return RLL_OK;
}

int rll_grid_export(rll_ctx* ctx, const rll_grid* g, uint64_t* keys, int32_t* cut, float* q, float* c)
{
    if (!ctx || !g) return RLL_E_INVALID;
    DeviceGuard dg(ctx->device);
    const size_t rows = (size_t)g->H * g->M;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (keys) e = cudaMemcpyAsync(keys, g->keys, 8 * (size_t)g->H, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && cut) e = cudaMemcpyAsync(cut, g->cut, 4 * rows, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "grid export");
    if (q || c) {
        float* w = (float*)ws_get(ctx, 8 * rows);
        if (!w) return RLL_E_NOMEM;
        int rc = grid_to_float(ctx, g, w, w + rows);
        if (rc != RLL_OK) return rc;
        if (q) e = cudaMemcpyAsync(q, w, 4 * rows, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && c) e = cudaMemcpyAsync(c, w + rows, 4 * rows, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return check_cuda(ctx, e, "grid export");
}

int rll_grid_import(rll_ctx* ctx, rll_grid* g, const uint64_t* keys, const int32_t* cut, const float* q, const float* c)
{
    if (!ctx || !g) return RLL_E_INVALID;
    if (!keys || !cut || !q || !c) return fail(ctx, RLL_E_INVALID, "grid import needs keys, cut, q and c");
    DeviceGuard dg(ctx->device);
    const size_t rows = (size_t)g->H * g->M;
    cudaStream_t s = ctx->stream;
    float* w = (float*)ws_get(ctx, 8 * rows);
    if (!w) return RLL_E_NOMEM;
    cudaError_t e = cudaMemcpyAsync(g->keys, keys, 8 * (size_t)g->H, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->cut, cut, 4 * rows, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, q, 4 * rows, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w + rows, c, 4 * rows, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "grid import");
    int rc = grid_from_float(ctx, g, w, w + rows);
    if (rc == RLL_OK) rc = grid_mark_occupied(ctx, g);
    if (rc != RLL_OK) return rc;
    return check_cuda(ctx, cudaStreamSynchronize(s), "grid import");
}

int rll_grid_destroy(rll_grid* grid)
{
    if (!grid) return RLL_OK;
    DeviceGuard g(grid->device);
    cudaDeviceSynchronize();
    free_grid(grid);
    return RLL_OK;
}

static int check_pass_args(rll_ctx* ctx, const rll_grid* grid, const rll_tree* tree, const float* pos,
                           const float* nrm, const float* albedo, int64_t n_points, const float* boxes,
                           int32_t n_boxes, int32_t spp, const float* rgb)
{
    if (!grid || !tree) return fail(ctx, RLL_E_INVALID, "grid / tree is NULL");
    if (grid->n_lights != tree->n) return fail(ctx, RLL_E_INVALID, "grid was created for another tree");
    if (n_points < 0) return fail(ctx, RLL_E_INVALID, "n_points < 0");
    if (spp < 1 || spp > 65536) return fail(ctx, RLL_E_INVALID, "spp must be in [1, 65536]");
    if ((uint64_t)n_points * (uint64_t)spp >= 0xFFFFFFFFull) return fail(ctx, RLL_E_INVALID, "n_points * spp must be < 2^32");
    if (n_boxes < 0 || n_boxes > kMaxBoxes) return fail(ctx, RLL_E_INVALID, "n_boxes must be in [0, 1024]");
    if (n_boxes > 0 && !boxes) return fail(ctx, RLL_E_INVALID, "boxes is NULL");
    if (n_points > 0 && (!pos || !nrm || !albedo || !rgb)) return fail(ctx, RLL_E_INVALID, "NULL G-buffer or rgb");
    return RLL_OK;
}

int rll_sample_and_shade_fp(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos, const float* nrm,
                            const float* albedo, const float* footprint, int64_t n_points, const float* boxes,
                            int32_t n_boxes, uint64_t seed, uint32_t frame, int32_t spp, float* rgb,
                            uint32_t* rec_key, float* rec_val, const rll_sample_debug* dbg)
{
    if (!ctx) return RLL_E_INVALID;
    int rc = check_pass_args(ctx, grid, tree, pos, nrm, albedo, n_points, boxes, n_boxes, spp, rgb);
    if (rc != RLL_OK) return rc;
    if ((rec_key == nullptr) != (rec_val == nullptr)) return fail(ctx, RLL_E_INVALID, "rec_key and rec_val go together");
    DeviceGuard g(ctx->device);
    return sample_and_shade(ctx, grid, tree, pos, nrm, albedo, footprint, n_points, boxes, n_boxes, seed, frame, spp,
                            rgb, rec_key, rec_val, dbg);
}

int rll_sample_and_shade_ex(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos, const float* nrm,
                            const float* albedo, int64_t n_points, const float* boxes, int32_t n_boxes,
                            uint64_t seed, uint32_t frame, int32_t spp, float* rgb, uint32_t* rec_key,
                            float* rec_val, const rll_sample_debug* dbg)
{
    return rll_sample_and_shade_fp(ctx, grid, tree, pos, nrm, albedo, nullptr, n_points, boxes, n_boxes, seed, frame,
                                   spp, rgb, rec_key, rec_val, dbg);
}

int rll_sample_and_shade(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos, const float* nrm,
                         const float* albedo, int64_t n_points, const float* boxes, int32_t n_boxes, uint64_t seed,
                         uint32_t frame, int32_t spp, float* rgb, uint32_t* rec_key, float* rec_val)
{
    return rll_sample_and_shade_ex(ctx, grid, tree, pos, nrm, albedo, n_points, boxes, n_boxes, seed, frame, spp,
                                   rgb, rec_key, rec_val, nullptr);
}

int rll_sample_power(rll_ctx* ctx, const rll_tree* tree, const float* pos, const float* nrm, const float* albedo,
                     int64_t n_points, const float* boxes, int32_t n_boxes, uint64_t seed, uint32_t frame,
                     int32_t spp, float* rgb, int32_t* light_out)
{
    if (!ctx) return RLL_E_INVALID;
    if (!tree) return fail(ctx, RLL_E_INVALID, "tree is NULL");
    if (n_points < 0 || spp < 1 || (uint64_t)n_points * (uint64_t)spp >= 0xFFFFFFFFull)
        return fail(ctx, RLL_E_INVALID, "bad n_points / spp");
    if (n_boxes < 0 || n_boxes > kMaxBoxes || (n_boxes > 0 && !boxes)) return fail(ctx, RLL_E_INVALID, "bad boxes");
    if (n_points > 0 && (!pos || !nrm || !albedo || !rgb)) return fail(ctx, RLL_E_INVALID, "NULL G-buffer or rgb");
    DeviceGuard g(ctx->device);
    return sample_power(ctx, tree, pos, nrm, albedo, n_points, boxes, n_boxes, seed, frame, spp, rgb, light_out);
}

int rll_learn_update(rll_ctx* ctx, rll_grid* grid, const uint32_t* rec_key, const float* rec_val, int64_t n_records)
{
    if (!ctx) return RLL_E_INVALID;
    if (!grid) return fail(ctx, RLL_E_INVALID, "grid is NULL");
    if (n_records < 0 || n_records >= 0xFFFFFFFFll) return fail(ctx, RLL_E_INVALID, "n_records out of range");
    if (n_records > 0 && (!rec_key || !rec_val)) return fail(ctx, RLL_E_INVALID, "NULL records");
    DeviceGuard g(ctx->device);
    return learn_update(ctx, grid, rec_key, rec_val, n_records);
}

int rll_learn_update_split(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const uint32_t* rec_key,
                           const float* rec_val, int64_t n_records)
{
    if (!ctx) return RLL_E_INVALID;
    if (!grid || !tree) return fail(ctx, RLL_E_INVALID, "grid / tree is NULL");
    if (grid->n_lights != tree->n) return fail(ctx, RLL_E_INVALID, "grid was created for another tree");
    if (n_records < 0 || n_records >= 0xFFFFFFFFll) return fail(ctx, RLL_E_INVALID, "n_records out of range");
    if (n_records > 0 && (!rec_key || !rec_val)) return fail(ctx, RLL_E_INVALID, "NULL records");
    DeviceGuard g(ctx->device);
    return learn_update_split(ctx, grid, tree, rec_key, rec_val, n_records);
}

int rll_split_collapse(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree)
{
    if (!ctx) return RLL_E_INVALID;
    if (!grid || !tree) return fail(ctx, RLL_E_INVALID, "grid / tree is NULL");
    if (grid->n_lights != tree->n) return fail(ctx, RLL_E_INVALID, "grid was created for another tree");
    DeviceGuard g(ctx->device);
    return split_collapse(ctx, grid, tree);
}

int rll_render_pass_host(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos, const float* nrm,
                         const float* albedo, int64_t n_points, const float* boxes, int32_t n_boxes, uint64_t seed,
                         uint32_t frame, int32_t spp, int32_t do_split, float* rgb)
{
    if (!ctx) return RLL_E_INVALID;
    int rc = check_pass_args(ctx, grid, tree, pos, nrm, albedo, n_points, boxes, n_boxes, spp, rgb);
    if (rc != RLL_OK) return rc;
    DeviceGuard g(ctx->device);
    const int64_t P = n_points, S = n_points * spp;
    auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t need = a(12 * P) * 3 + a(4 * P) + a(24 * (size_t)std::max(n_boxes, 1)) + a(4 * S) * 2;
    if (need > ctx->stage_bytes) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        if (cudaMalloc(&ctx->stage, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, RLL_E_NOMEM, "cannot allocate staging buffers");
        }
        ctx->stage_bytes = need;
    }
    if (!ctx->pipe_ready) {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->down, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->comp2, cudaStreamNonBlocking);
        for (cudaEvent_t& ev : ctx->ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return check_cuda(ctx, e, "render_pass_host: streams");
        ctx->pipe_ready = true;
    }
    char* w = (char*)ctx->stage;
    float* d_pos = (float*)w; w += a(12 * P);
    float* d_nrm = (float*)w; w += a(12 * P);
    float* d_rgb = (float*)w; w += a(12 * P);
    float* d_alb = (float*)w; w += a(4 * P);
    float* d_box = (float*)w; w += a(24 * (size_t)std::max(n_boxes, 1));
    uint32_t* d_key = (uint32_t*)w; w += a(4 * S);
    float* d_val = (float*)w;

    // Host memory the device can address (page-locked and mapped, as every cudaHostAlloc /
    // cudaHostRegister allocation is under unified addressing): the sampling kernel reads the
    // G-buffer and writes rgb over the host link itself; only the boxes are copied.
    auto mapped = [](const void* p) -> void* {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
    };
    if (ctx->host_zero_copy) {
        void *zp = mapped(pos), *zn = mapped(nrm), *za = mapped(albedo), *zr = mapped(rgb);
        if (zp && zn && za && zr) {
            cudaStream_t s = ctx->stream;
            cudaError_t e = cudaSuccess;
            if (n_boxes > 0) e = cudaMemcpyAsync(d_box, boxes, 24 * (size_t)n_boxes, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return check_cuda(ctx, e, "render_pass_host: boxes");
            rc = sample_and_shade(ctx, grid, tree, (const float*)zp, (const float*)zn, (const float*)za, nullptr, P,
                                  d_box, n_boxes, seed, frame, spp, (float*)zr, d_key, d_val, nullptr);
            if (rc == RLL_OK)
                rc = do_split ? learn_update_split(ctx, grid, tree, d_key, d_val, S)
                              : learn_update(ctx, grid, d_key, d_val, S);
            e = cudaStreamSynchronize(s);  // rgb is complete in host memory after this
            if (rc != RLL_OK) return rc;
            return check_cuda(ctx, e, "render_pass_host");
        }
    }

    // Copy/compute overlap: the points are cut into chunks (sizes below); chunk k is
    // uploaded on `up`, shaded on the main stream or comp2 (alternately, so a
    // chunk's tail overlaps the next chunk's start) once its upload is done,
    // and its rgb read back on `down` once it is shaded. Learning and
    // split-collapse follow all chunks on the main stream and overlap the
    // last read-backs. Sample ids, records and rgb are those of one launch.
    // Chunk sizes grow by 3/2 (multiples of 256 points, at least 4 096): the first upload, which
    // nothing overlaps, is short, and an upload (28 B a point) still ends before the shading of
    // the chunk ahead of it.
    const int want = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->host_chunks, RLL_HOST_MAX_CHUNKS));
    int64_t bnd[RLL_HOST_MAX_CHUNKS + 1];
    int nc = 0;
    {
        double wsum = 0.0, w = 1.0;
        for (int k = 0; k < want; ++k, w *= 1.5) wsum += w;
        int64_t b = 0;
        w = 1.0;
        bnd[0] = 0;
        for (int k = 0; k < want && b < P; ++k, w *= 1.5) {
            int64_t len = (int64_t)((double)P * w / wsum);
            len = std::max<int64_t>(4096, (len + 255) & ~(int64_t)255);
            b = (k == want - 1) ? P : std::min<int64_t>(P, b + len);
            bnd[++nc] = b;
        }
    }
    cudaStream_t s = ctx->stream, sc[2] = {ctx->stream, ctx->comp2};
    cudaEvent_t* ev_up = ctx->ev;
    cudaEvent_t* ev_done = ctx->ev + RLL_HOST_MAX_CHUNKS;
    cudaEvent_t ev_start = ctx->ev[2 * RLL_HOST_MAX_CHUNKS], ev_join = ctx->ev[2 * RLL_HOST_MAX_CHUNKS + 1],
                ev_down = ctx->ev[2 * RLL_HOST_MAX_CHUNKS + 2];
    // planes of [3][P] arrays: one strided copy per chunk where the pitch allows
    auto planes = [&](float* dst, const float* src, int64_t b, int64_t n, cudaMemcpyKind kind, cudaStream_t st) {
        const size_t pitch = 4 * (size_t)P;
        if (pitch <= (size_t)INT32_MAX)
            return cudaMemcpy2DAsync(dst + b, pitch, src + b, pitch, 4 * (size_t)n, 3, kind, st);
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(dst + k * P + b, src + k * P + b, 4 * (size_t)n, kind, st);
        return e;
    };
    // the boxes and their sorted copy first (both compute streams wait for them)
    cudaError_t e = cudaSuccess;
    if (n_boxes > 0) e = cudaMemcpyAsync(d_box, boxes, 24 * (size_t)n_boxes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "render_pass_host: boxes");
    const void* sorted = nullptr;
    rc = sort_boxes(ctx, d_box, n_boxes, s, &sorted);
    if (rc != RLL_OK) return rc;
    e = cudaEventRecord(ev_start, s);  // the grid's earlier updates come first
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->comp2, ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->down, ev_start, 0);
    for (int k = 0; k < nc && e == cudaSuccess && rc == RLL_OK; ++k) {
        const int64_t b = bnd[k], n = bnd[k + 1] - bnd[k];
        e = planes(d_pos, pos, b, n, cudaMemcpyHostToDevice, ctx->up);
        if (e == cudaSuccess) e = planes(d_nrm, nrm, b, n, cudaMemcpyHostToDevice, ctx->up);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_alb + b, albedo + b, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->up);
        if (e == cudaSuccess) e = cudaEventRecord(ev_up[k], ctx->up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sc[k & 1], ev_up[k], 0);
        if (e != cudaSuccess) break;
        rc = rll::sample_and_shade_range(ctx, grid, tree, d_pos, d_nrm, d_alb, nullptr, P, b, b + n, d_box, n_boxes,
                                         seed, frame, spp, d_rgb, d_key, d_val, nullptr, sc[k & 1], sorted);
        if (rc != RLL_OK) break;
        e = cudaEventRecord(ev_done[k], sc[k & 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->down, ev_done[k], 0);
        if (e == cudaSuccess) e = planes(rgb, d_rgb, b, n, cudaMemcpyDeviceToHost, ctx->down);
    }
    if (e == cudaSuccess && rc == RLL_OK) {
        e = cudaEventRecord(ev_join, ctx->comp2);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join, 0);
    }
    if (e == cudaSuccess && rc == RLL_OK)
        rc = do_split ? learn_update_split(ctx, grid, tree, d_key, d_val, S) : learn_update(ctx, grid, d_key, d_val, S);
    if (e == cudaSuccess) e = cudaEventRecord(ev_down, ctx->down);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_down, 0);
    // every stream of the pipeline is drained before returning, also on errors
    cudaError_t e2 = cudaStreamSynchronize(ctx->up);
    cudaError_t e3 = cudaStreamSynchronize(ctx->comp2);
    cudaError_t e4 = cudaStreamSynchronize(ctx->down);
    cudaError_t e5 = cudaStreamSynchronize(s);
    if (rc != RLL_OK) return rc;
    for (cudaError_t x : {e2, e3, e4, e5})
        if (e == cudaSuccess) e = x;
    return check_cuda(ctx, e, "render_pass_host");
}

}  // extern "C"
