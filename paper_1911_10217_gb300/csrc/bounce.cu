// Path vertices of one diffuse bounce and their footprints (Section 3, first
// ingredient: the cells of a path vertex are sized from its ray footprint,
// derived from the vertex's area pdf).
//
// One thread per shading point x (unit normal n), occluder boxes staged in
// shared memory once per block:
//   a uniform point (a, b) of the unit disk by rejection from the point's
//   Philox stream (counter (point, frame, draw / 4, 1); pair k = draws 2k,
//   2k + 1 as 2u - 1; first k < 16 inside the disk, else the centre);
//   lifted to the hemisphere about n (Malley): d = a u + b v + sqrt(1 - a^2 -
//   b^2) n, tangents u = normalise(n x t), v = n x u, t = x axis unless
//   |n.x| >= 0.9, then z axis;
//   the nearest surface ahead of x + 1e-4 n: a wall of the room (from the
//   inside) or a box face (slab test), t > 1e-6;
//   y = o + t d, its face normal turned toward x, and the footprint
//   f = t sqrt(pi / (N_t cos_x cos_y)) = (N_t p_A)^(-1/2), p_A = cos_x cos_y
//   / (pi t^2) the area density of y for one path, shared by the N_t paths
//   that leave one tile; a ray with nothing ahead escapes (y = o, normal 0,
//   f = +inf).
// Every step is one correctly rounded binary32 operation (no contraction),
// so the hit face, a decision, is reproducible.
#include <cuda_runtime.h>

#include "rll_device.cuh"
#include "rll_internal.h"
#include "sample_core.cuh"

namespace rll {
namespace {

constexpr int kBounceThreads = 256;
constexpr int kBounceTries = 16;
constexpr float kBounceOffset = 1e-4f;
constexpr float kBounceTmin = 1e-6f;
constexpr float kPiF = 3.14159265358979323846f;

__device__ __forceinline__ float fdivr(float a, float b) { return __fdiv_rn(a, b); }

__global__ void __launch_bounds__(kBounceThreads)
k_bounce(const float* __restrict__ pos, const float* __restrict__ nrm, int64_t np, const float* __restrict__ boxes,
         int n_boxes, float r0, float r1, float r2, float r3, float r4, float r5, uint2 key, uint32_t frame,
         float paths_per_tile, float* __restrict__ y_out, float* __restrict__ ny_out, float* __restrict__ fp_out)
{
    extern __shared__ float4 s_box[];
    stage_boxes(s_box, boxes, n_boxes);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const float x[3] = {pos[p], pos[np + p], pos[2 * np + p]};
    const float n[3] = {nrm[p], nrm[np + p], nrm[2 * np + p]};

    // the disk point
    float a = 0.0f, b = 0.0f;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    for (int k = 0; k < kBounceTries; ++k) {
        if ((k & 1) == 0) w = philox4x32_10(make_uint4((uint32_t)p, frame, (uint32_t)(k >> 1), 1u), key);
        const float ua = u24((k & 1) ? w.z : w.x), ub = u24((k & 1) ? w.w : w.y);
        const float ta = fsub(fmul(2.0f, ua), 1.0f), tb = fsub(fmul(2.0f, ub), 1.0f);
        if (fadd(fmul(ta, ta), fmul(tb, tb)) < 1.0f) {
            a = ta;
            b = tb;
            break;
        }
    }
    const float s = fadd(fmul(a, a), fmul(b, b));
    const float c = __fsqrt_rn(fmaxf(0.0f, fsub(1.0f, s)));  // cos(theta_x)

    // tangent frame of n
    const bool tx = fabsf(n[0]) < 0.9f;
    const float t0 = tx ? 1.0f : 0.0f, t2 = tx ? 0.0f : 1.0f;
    float u[3] = {fsub(fmul(n[1], t2), fmul(n[2], 0.0f)), fsub(fmul(n[2], t0), fmul(n[0], t2)),
                  fsub(fmul(n[0], 0.0f), fmul(n[1], t0))};
    const float ul = __fsqrt_rn(fadd(fadd(fmul(u[0], u[0]), fmul(u[1], u[1])), fmul(u[2], u[2])));
    for (int k = 0; k < 3; ++k) u[k] = fdivr(u[k], ul);
    const float v[3] = {fsub(fmul(n[1], u[2]), fmul(n[2], u[1])), fsub(fmul(n[2], u[0]), fmul(n[0], u[2])),
                        fsub(fmul(n[0], u[1]), fmul(n[1], u[0]))};

    float d[3], o[3], inv[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = fadd(fadd(fmul(a, u[k]), fmul(b, v[k])), fmul(c, n[k]));
        o[k] = fadd(x[k], fmul(kBounceOffset, n[k]));
        inv[k] = fdivr(1.0f, d[k]);
    }

    // the first room wall ahead
    const float rlo[3] = {r0, r1, r2}, rhi[3] = {r3, r4, r5};
    float t_best = INFINITY;
    int axis = 0;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0f) continue;
        const float wall = d[k] > 0.0f ? rhi[k] : rlo[k];
        const float t = fmul(fsub(wall, o[k]), inv[k]);
        if (t > kBounceTmin && t < t_best) {
            t_best = t;
            axis = k;
        }
    }
    // the nearest box face in front of it
    for (int i = 0; i < n_boxes; ++i) {
        const float4 lo4 = s_box[2 * i], hi4 = s_box[2 * i + 1];
        const float blo[3] = {lo4.x, lo4.y, lo4.z}, bhi[3] = {hi4.x, hi4.y, hi4.z};
        float tn = -INFINITY, tf = INFINITY;
        int ax = 0;
        bool miss = false;
        for (int k = 0; k < 3; ++k) {
            if (d[k] == 0.0f) {  // parallel to this slab: inside it or a miss
                if (!(o[k] > blo[k] && o[k] < bhi[k])) miss = true;
                continue;
            }
            const float ta = fmul(fsub(blo[k], o[k]), inv[k]);
            const float tb = fmul(fsub(bhi[k], o[k]), inv[k]);
            const float lo = fminf(ta, tb), hi = fmaxf(ta, tb);
            if (lo > tn) {
                tn = lo;
                ax = k;
            }
            tf = fminf(tf, hi);
        }
        if (!miss && tn < tf && tn > kBounceTmin && tn < t_best) {
            t_best = tn;
            axis = ax;
        }
    }
    if (t_best == INFINITY) {  // nothing ahead: the path escapes
        for (int k = 0; k < 3; ++k) {
            y_out[k * np + p] = o[k];
            ny_out[k * np + p] = 0.0f;
        }
        fp_out[p] = INFINITY;
        return;
    }
    for (int k = 0; k < 3; ++k) {
        y_out[k * np + p] = fadd(o[k], fmul(t_best, d[k]));
        ny_out[k * np + p] = k == axis ? (d[axis] > 0.0f ? -1.0f : 1.0f) : 0.0f;
    }
    const float cy = fabsf(d[axis]);  // cos(theta_y)
    const float q = fmul(fmul(paths_per_tile, fmaxf(c, 1e-6f)), fmaxf(cy, 1e-6f));
    fp_out[p] = fmul(t_best, __fsqrt_rn(fdivr(kPiF, q)));
}

}  // namespace
}  // namespace rll

extern "C" int rll_bounce_vertices(rll_ctx* ctx, const float* pos, const float* nrm, int64_t n_points,
                                   const float* boxes, int32_t n_boxes, const float* room, uint64_t seed,
                                   uint32_t frame, float paths_per_tile, float* out_pos, float* out_nrm,
                                   float* out_footprint)
{
    using namespace rll;
    if (!ctx) return RLL_E_INVALID;
    if (n_points < 0 || n_points > 0xFFFFFFFFll) return fail(ctx, RLL_E_INVALID, "n_points must be in [0, 2^32)");
    if (n_boxes < 0 || n_boxes > kMaxBoxes || (n_boxes > 0 && !boxes))
        return fail(ctx, RLL_E_INVALID, "n_boxes must be in [0, 1024] with boxes given");
    if (!room) return fail(ctx, RLL_E_INVALID, "room is NULL");
    if (!(paths_per_tile > 0.0f) || !std::isfinite(paths_per_tile))
        return fail(ctx, RLL_E_INVALID, "paths_per_tile must be > 0");
    if (n_points > 0 && (!pos || !nrm || !out_pos || !out_nrm || !out_footprint))
        return fail(ctx, RLL_E_INVALID, "NULL point or output array");
    if (n_points == 0) return RLL_OK;
    DeviceGuard g(ctx->device);
    const unsigned blocks = (unsigned)((n_points + kBounceThreads - 1) / kBounceThreads);
    const size_t smem = sizeof(float4) * 2 * (size_t)(n_boxes > 0 ? n_boxes : 1);
    k_bounce<<<blocks, kBounceThreads, smem, ctx->stream>>>(
        pos, nrm, n_points, boxes, n_boxes, room[0], room[1], room[2], room[3], room[4], room[5],
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), frame, paths_per_tile, out_pos, out_nrm, out_footprint);
    return check_cuda(ctx, cudaGetLastError(), "bounce kernel");
}
