// Light tree build (Section 3: sort all lights and build one binary tree over
// them; Section 3.1: an LBVH over the 3-d light positions).
//
//   centroids + scene box -> 30-bit Morton codes -> stable radix sort
//   (ties by input index) -> binary radix tree over (code << 32 | index)
//   (Karras, HPG 2012: one thread per internal node, no recursion) ->
//   leaf records -> bottom-up bounds (atomic arrival counter per node, the
//   second child to arrive finishes its parent) -> cone axis -> cone cosine
//   minimum over each node's lights (one thread per light walks to the root)
//   -> child-pair records for the descent -> prefix sum of leaf power.
#include <cuda_runtime.h>

#include "rll_device.cuh"
#include "rll_internal.h"

namespace rll {
namespace {

constexpr int kBlock = 256;

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

__global__ void k_bbox_init(int* bbox)
{
    if (threadIdx.x < 3) bbox[threadIdx.x] = float_to_ordered(INFINITY);
    else if (threadIdx.x < 6) bbox[threadIdx.x] = float_to_ordered(-INFINITY);
}

__device__ __forceinline__ float centroid(const float* v, int k)
{
    return fdiv(fadd(fadd(v[k], v[3 + k]), v[6 + k]), 3.0f);
}

__global__ void k_centroid_bbox(const float* __restrict__ tri, int64_t n, int* __restrict__ bbox)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < n) {
        const float* v = tri + i * 9;
        for (int k = 0; k < 3; ++k) {
            const float c = centroid(v, k);
            lo[k] = c;
            hi[k] = c;
        }
    }
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bbox[k], float_to_ordered(lo[k]));
            atomicMax(&bbox[3 + k], float_to_ordered(hi[k]));
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(const float* __restrict__ tri, int64_t n, const int* __restrict__ bbox,
                         uint32_t* __restrict__ codes, uint32_t* __restrict__ idx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* v = tri + i * 9;
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        const float lo = ordered_to_float(bbox[k]), hi = ordered_to_float(bbox[3 + k]);
        const float ext = fsub(hi, lo);
        const float u = ext > 0.0f ? fdiv(fsub(centroid(v, k), lo), ext) : 0.0f;
        float f = floorf(fmul(u, 1024.0f));
        f = fminf(fmaxf(f, 0.0f), 1023.0f);
        q[k] = (uint32_t)f;
    }
    codes[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    idx[i] = (uint32_t)i;
}

__device__ __forceinline__ int delta(const uint32_t* codes, const uint32_t* idx, int64_t n, int64_t i, int64_t j)
{
    if (j < 0 || j >= n) return -1;
    const unsigned long long a = ((unsigned long long)codes[i] << 32) | idx[i];
    const unsigned long long b = ((unsigned long long)codes[j] << 32) | idx[j];
    return __clzll((long long)(a ^ b));
}

__global__ void k_karras(const uint32_t* __restrict__ codes, const uint32_t* __restrict__ idx, int64_t n,
                         int32_t* __restrict__ left, int32_t* __restrict__ right, int32_t* __restrict__ parent,
                         uint32_t* __restrict__ begin, uint32_t* __restrict__ end)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(codes, idx, n, i, i + 1) - delta(codes, idx, n, i, i - 1)) > 0 ? 1 : -1;
    const int dmin = delta(codes, idx, n, i, i - d);
    int64_t lmax = 2;
    while (delta(codes, idx, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, idx, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(codes, idx, n, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(codes, idx, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t g = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    const int32_t a = (lo == g) ? (int32_t)(n - 1 + g) : (int32_t)g;
    const int32_t c = (hi == g + 1) ? (int32_t)(n - 1 + g + 1) : (int32_t)(g + 1);
    left[i] = a;
    right[i] = c;
    parent[a] = (int32_t)i;
    parent[c] = (int32_t)i;
    begin[i] = (uint32_t)lo;
    end[i] = (uint32_t)(hi + 1);
}

__device__ __forceinline__ void cross32(const float* v, float cr[3], float* len)
{
    const float e1x = fsub(v[3], v[0]), e1y = fsub(v[4], v[1]), e1z = fsub(v[5], v[2]);
    const float e2x = fsub(v[6], v[0]), e2y = fsub(v[7], v[1]), e2z = fsub(v[8], v[2]);
    cr[0] = fsub(fmul(e1y, e2z), fmul(e1z, e2y));
    cr[1] = fsub(fmul(e1z, e2x), fmul(e1x, e2z));
    cr[2] = fsub(fmul(e1x, e2y), fmul(e1y, e2x));
    *len = fsqrt(fadd(fadd(fmul(cr[0], cr[0]), fmul(cr[1], cr[1])), fmul(cr[2], cr[2])));
}

__global__ void k_leaves(const float* __restrict__ tri, const float* __restrict__ emis, int64_t n,
                         const uint32_t* __restrict__ sorted_idx, uint32_t* __restrict__ perm,
                         LightRec* __restrict__ lights, NodeRec* __restrict__ nodes,
                         float* __restrict__ axis_sum)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const uint32_t i = sorted_idx[l];
    perm[l] = i;
    const float* v = tri + (int64_t)i * 9;
    const float* le = emis + (int64_t)i * 3;
    float cr[3], len;
    cross32(v, cr, &len);
    const float area = fmul(0.5f, len);
    LightRec L;
    NodeRec R;
    for (int k = 0; k < 3; ++k) {
        L.v0[k] = v[k];
        L.v1[k] = v[3 + k];
        L.v2[k] = v[6 + k];
        L.le[k] = le[k];
        L.n[k] = fdiv(cr[k], len);
        R.bmin[k] = fminf(fminf(v[k], v[3 + k]), v[6 + k]);
        R.bmax[k] = fmaxf(fmaxf(v[k], v[3 + k]), v[6 + k]);
        R.axis[k] = 0.0f;
    }
    L.area = area;
    const float lum = fadd(fadd(fmul(0.2126f, le[0]), fmul(0.7152f, le[1])), fmul(0.0722f, le[2]));
    R.phi = fmul(lum, area);
    R.cos_t = 1.0f;
    const int64_t id = n - 1 + l;
    R.id = (uint32_t)id;
    R.begin = (uint32_t)l;
    R.end = (uint32_t)(l + 1);
    lights[l] = L;
    nodes[id] = R;
    axis_sum[id * 3 + 0] = cr[0];
    axis_sum[id * 3 + 1] = cr[1];
    axis_sum[id * 3 + 2] = cr[2];
}

__device__ __forceinline__ NodeRec load_node_cg(const NodeRec* p)
{
    NodeRec r;
    const float4* s = reinterpret_cast<const float4*>(p);
    float4* d = reinterpret_cast<float4*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = __ldcg(s + k);
    return r;
}

__global__ void k_bottom_up(int64_t n, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                            const int32_t* __restrict__ parent, NodeRec* nodes, float* axis_sum,
                            uint32_t* counters)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    int64_t node = n - 1 + l;
    int32_t p = parent[node];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&counters[p], 1u) == 0u) return;  // the sibling finishes p
        __threadfence();
        const int32_t a = left[p], c = right[p];
        const NodeRec A = load_node_cg(nodes + a), Cn = load_node_cg(nodes + c);
        NodeRec R;
        for (int k = 0; k < 3; ++k) {
            R.bmin[k] = fminf(A.bmin[k], Cn.bmin[k]);
            R.bmax[k] = fmaxf(A.bmax[k], Cn.bmax[k]);
            R.axis[k] = 0.0f;
            axis_sum[(int64_t)p * 3 + k] =
                fadd(__ldcg(axis_sum + (int64_t)a * 3 + k), __ldcg(axis_sum + (int64_t)c * 3 + k));
        }
        R.phi = fadd(A.phi, Cn.phi);
        R.cos_t = 1.0f;
        R.id = (uint32_t)p;
        R.begin = A.begin;
        R.end = Cn.end;
        nodes[p] = R;
        node = p;
        p = parent[p];
    }
}

__global__ void k_axis(int64_t nn, NodeRec* __restrict__ nodes, const float* __restrict__ axis_sum,
                       int* __restrict__ cosmin)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const float sx = axis_sum[i * 3], sy = axis_sum[i * 3 + 1], sz = axis_sum[i * 3 + 2];
    const float len = fsqrt(fadd(fadd(fmul(sx, sx), fmul(sy, sy)), fmul(sz, sz)));
    NodeRec& r = nodes[i];
    if (len > 0.0f) {
        r.axis[0] = fdiv(sx, len);
        r.axis[1] = fdiv(sy, len);
        r.axis[2] = fdiv(sz, len);
        cosmin[i] = float_to_ordered(1.0f);
    } else {
        r.axis[0] = 0.0f;
        r.axis[1] = 0.0f;
        r.axis[2] = 1.0f;
        cosmin[i] = float_to_ordered(-1.0f);
    }
}

__global__ void k_cone(int64_t n, const LightRec* __restrict__ lights, const NodeRec* __restrict__ nodes,
                       const int32_t* __restrict__ parent, int* __restrict__ cosmin)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const float nx = lights[l].n[0], ny = lights[l].n[1], nz = lights[l].n[2];
    int64_t node = n - 1 + l;
    int guard = 0;
    while (node >= 0 && guard++ < kMaxTreeDepth) {
        const NodeRec& r = nodes[node];
        const float d = fadd(fadd(fmul(r.axis[0], nx), fmul(r.axis[1], ny)), fmul(r.axis[2], nz));
        atomicMin(&cosmin[node], float_to_ordered(d));
        node = parent[node];
    }
}

__global__ void k_finalize(int64_t nn, NodeRec* __restrict__ nodes, const int* __restrict__ cosmin)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    nodes[i].cos_t = fmaxf(-1.0f, ordered_to_float(cosmin[i]));
}

__global__ void k_pairs(int64_t n, const NodeRec* __restrict__ nodes, const int32_t* __restrict__ left,
                        const int32_t* __restrict__ right, PairRec* __restrict__ pairs, float* __restrict__ leaf_phi)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n - 1) {
        const DescRec L = make_desc(nodes[left[i]]), R = make_desc(nodes[right[i]]);
        PairRec q;
        q.c0 = make_float2(L.c[0], R.c[0]);
        q.c1 = make_float2(L.c[1], R.c[1]);
        q.c2 = make_float2(L.c[2], R.c[2]);
        q.r = make_float2(L.r, R.r);
        q.phi = make_float2(L.phi, R.phi);
        q.a0 = make_float2(L.axis[0], R.axis[0]);
        q.a1 = make_float2(L.axis[1], R.axis[1]);
        q.a2 = make_float2(L.axis[2], R.axis[2]);
        {  // exact: 1 - cos theta and sin theta are binary16 numbers
            const __half2 hl = __halves2half2(__float2half_rn(fsub(1.0f, L.cos_t)), __float2half_rn(L.sin_t));
            const __half2 hr = __halves2half2(__float2half_rn(fsub(1.0f, R.cos_t)), __float2half_rn(R.sin_t));
            q.cs = make_uint2(*reinterpret_cast<const uint32_t*>(&hl), *reinterpret_cast<const uint32_t*>(&hr));
        }
        q.id = make_uint2(L.id, R.id);
        pairs[i] = q;
    }
    if (i < n) leaf_phi[i] = nodes[n - 1 + i].phi;
}

// candidates of the two-level descent below internal node i, in light order
__global__ void k_quads(int64_t n, const NodeRec* __restrict__ nodes, const int32_t* __restrict__ left,
                        const int32_t* __restrict__ right, DescRec* __restrict__ quads)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int32_t cand[4];
    int k = 0;
    const int32_t kids[2] = {left[i], right[i]};
    for (int j = 0; j < 2; ++j) {
        const int32_t x = kids[j];
        if ((int64_t)x >= n - 1) {
            cand[k++] = x;
        } else {
            cand[k++] = left[x];
            cand[k++] = right[x];
        }
    }
    for (int j = 0; j < 4; ++j) {
        DescRec d{};
        if (j < k) d = make_desc(nodes[cand[j]]);
        else d.id = 0xFFFFFFFFu;
        quads[4 * i + j] = d;
    }
}

__global__ void k_update_emission(int64_t n, const uint32_t* __restrict__ perm, const float* __restrict__ emis,
                                  LightRec* __restrict__ lights)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const uint32_t i = perm[l];
    lights[l].le[0] = emis[(int64_t)i * 3];
    lights[l].le[1] = emis[(int64_t)i * 3 + 1];
    lights[l].le[2] = emis[(int64_t)i * 3 + 2];
}

// ---------------------------------------------------------------- SAOH split positions
// Surface-area-orientation split positions over the Morton order (Section
// 3.1 names a hierarchy that considers orientations and a surface area
// heuristic as future work): every node stays a contiguous range of the
// sorted lights; its split position is the candidate (every position when
// the range has at most 17 lights, else the 15 positions b + floor(m j /
// 16) and the Morton split) of least cost(L) + cost(R), ties to the
// smallest, with cost(S) = phi(S) * SA(box(S)) * (2 - |sum c| / sum |c|),
// c the winding cross product of a light. phi, |c| and c are summed exactly
// in 64-bit fixed point (scale 2^(30 - e), e the exponent of the largest
// value), so the sums do not depend on the summation order; the cost is
// binary32 from the sums converted to float. Internal node id = (split
// position - the root's) mod (n - 1): root 0. Built one level per launch,
// one block per node.

// fixed-point values of light l: phi, |c|, c (5 int64 arrays of n + 1, entry l + 1)
__global__ void k_saoh_max(int64_t n, const NodeRec* __restrict__ nodes, const float* __restrict__ axis_sum,
                           int* __restrict__ mx)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float mphi = 0.0f, mc = 0.0f;
    if (l < n) {
        const int64_t id = n - 1 + l;
        mphi = nodes[id].phi;
        const float cx = axis_sum[id * 3], cy = axis_sum[id * 3 + 1], cz = axis_sum[id * 3 + 2];
        const float len = fsqrt(fadd(fadd(fmul(cx, cx), fmul(cy, cy)), fmul(cz, cz)));
        mc = fmaxf(fmaxf(fabsf(cx), fabsf(cy)), fmaxf(fabsf(cz), len));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mphi = fmaxf(mphi, __shfl_xor_sync(0xffffffffu, mphi, o));
        mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(mx, __float_as_int(mphi));  // non-negative floats order as integers
        atomicMax(mx + 1, __float_as_int(mc));
    }
}

__device__ __forceinline__ int exponent_of(float v)  // v = f * 2^e, f in [0.5, 1); 0 -> 0
{
    if (!(v > 0.0f)) return 0;
    int e;
    frexpf(v, &e);
    return e;
}

__global__ void k_saoh_fixed(int64_t n, const NodeRec* __restrict__ nodes, const float* __restrict__ axis_sum,
                             const int* __restrict__ mx, long long* __restrict__ fx)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l > n) return;
    const int64_t stride = n + 1;
    if (l == 0) {
        for (int k = 0; k < 5; ++k) fx[k * stride] = 0;
        return;
    }
    const int64_t id = n - 1 + (l - 1);
    const int sp = 30 - exponent_of(__int_as_float(mx[0])), sc = 30 - exponent_of(__int_as_float(mx[1]));
    const float cx = axis_sum[id * 3], cy = axis_sum[id * 3 + 1], cz = axis_sum[id * 3 + 2];
    const float len = fsqrt(fadd(fadd(fmul(cx, cx), fmul(cy, cy)), fmul(cz, cz)));
    fx[l] = __double2ll_rn(ldexp((double)nodes[id].phi, sp));
    fx[stride + l] = __double2ll_rn(ldexp((double)len, sc));
    fx[2 * stride + l] = __double2ll_rn(ldexp((double)cx, sc));
    fx[3 * stride + l] = __double2ll_rn(ldexp((double)cy, sc));
    fx[4 * stride + l] = __double2ll_rn(ldexp((double)cz, sc));
}

// inclusive prefix sums of the 5 arrays (n + 1 entries each), in place: one
// block per array, chunks of 1024 carried sequentially (exact integers)
__global__ void __launch_bounds__(1024) k_saoh_scan(int64_t n, long long* __restrict__ fx)
{
    __shared__ long long s_w[32];
    long long* a = fx + (int64_t)blockIdx.x * (n + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry = 0;
    for (int64_t base = 0; base <= n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        long long v = i <= n ? a[i] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) s_w[warp] = v;
        __syncthreads();
        if (warp == 0) {
            long long w = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const long long incl = v + (warp > 0 ? s_w[warp - 1] : 0) + carry;
        if (i <= n) a[i] = incl;
        carry += s_w[31];
        __syncthreads();
    }
}

struct SaohNode {
    uint32_t b, e;       // range [b, e), e - b >= 2
    int32_t parent;      // -1 at the root
    uint32_t side;       // 0: left child of parent, 1: right
};

__device__ __forceinline__ float box_area(const float lo[3], const float hi[3])
{
    const float dx = fsub(hi[0], lo[0]), dy = fsub(hi[1], lo[1]), dz = fsub(hi[2], lo[2]);
    return fmul(2.0f, fadd(fadd(fmul(dx, dy), fmul(dy, dz)), fmul(dz, dx)));
}

__device__ __forceinline__ float saoh_cost(const long long* fx, int64_t n, uint32_t lo, uint32_t hi,
                                           const float blo[3], const float bhi[3])
{
    const int64_t st = n + 1;
    const float phi = __ll2float_rn(fx[hi] - fx[lo]);
    const float area = __ll2float_rn(fx[st + hi] - fx[st + lo]);
    const float cx = __ll2float_rn(fx[2 * st + hi] - fx[2 * st + lo]);
    const float cy = __ll2float_rn(fx[3 * st + hi] - fx[3 * st + lo]);
    const float cz = __ll2float_rn(fx[4 * st + hi] - fx[4 * st + lo]);
    float om = 1.0f;
    if (area > 0.0f) om = fsub(2.0f, fdiv(fsqrt(fadd(fadd(fmul(cx, cx), fmul(cy, cy)), fmul(cz, cz))), area));
    return fmul(fmul(phi, box_area(blo, bhi)), om);
}

constexpr int kSaohThreads = 128;
constexpr int kSaohCand = 17;

__global__ void __launch_bounds__(kSaohThreads)
k_saoh_level(int64_t n, const SaohNode* __restrict__ in, uint32_t count, SaohNode* __restrict__ out,
             uint32_t* __restrict__ out_count, const uint32_t* __restrict__ codes, const uint32_t* __restrict__ idx,
             const NodeRec* __restrict__ nodes, const long long* __restrict__ fx, int64_t* __restrict__ groot,
             int32_t* __restrict__ left, int32_t* __restrict__ right, int32_t* __restrict__ parent)
{
    __shared__ uint32_t s_bound[kSaohCand + 2];  // b, sorted candidates, e
    __shared__ int s_nb;
    __shared__ int s_box[kSaohCand + 1][6];      // ordered-int min xyz, max xyz per segment
    const uint32_t w = blockIdx.x;
    if (w >= count) return;
    const SaohNode nd = in[w];
    const uint32_t b = nd.b, e = nd.e, m = e - b;
    if (threadIdx.x == 0) {
        uint32_t c[kSaohCand];
        int nc = 0;
        if (m <= 17) {
            for (uint32_t k = b + 1; k < e; ++k) c[nc++] = k;
        } else {
            // Morton split: last j in [b, e-2] sharing a longer prefix with b than e-1 does
            const unsigned long long kb = ((unsigned long long)codes[b] << 32) | idx[b];
            const unsigned long long ke = ((unsigned long long)codes[e - 1] << 32) | idx[e - 1];
            const int prefix = __clzll((long long)(kb ^ ke));
            uint32_t lo = b, hi = e - 2;  // invariant: lo qualifies (lo == b always does)
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo + 1) / 2;
                const unsigned long long km = ((unsigned long long)codes[mid] << 32) | idx[mid];
                if (__clzll((long long)(kb ^ km)) > prefix) lo = mid;
                else hi = mid - 1;
            }
            const uint32_t kmort = lo + 1;
            bool dup = false;
            for (int j = 1; j <= 15; ++j) {
                c[nc] = b + (uint32_t)(((uint64_t)m * (uint64_t)j) / 16u);
                dup |= c[nc] == kmort;
                ++nc;
            }
            if (!dup) c[nc++] = kmort;
            for (int i = 1; i < nc; ++i) {  // sort ascending
                const uint32_t v = c[i];
                int j = i - 1;
                while (j >= 0 && c[j] > v) {
                    c[j + 1] = c[j];
                    --j;
                }
                c[j + 1] = v;
            }
        }
        s_bound[0] = b;
        for (int i = 0; i < nc; ++i) s_bound[i + 1] = c[i];
        s_bound[nc + 1] = e;
        s_nb = nc + 2;
    }
    for (int i = threadIdx.x; i < (kSaohCand + 1) * 6; i += blockDim.x)
        s_box[i / 6][i % 6] = float_to_ordered(i % 6 < 3 ? INFINITY : -INFINITY);
    __syncthreads();
    const int nb = s_nb;
    for (uint32_t l = b + threadIdx.x; l < e; l += blockDim.x) {
        int lo = 0, hi = nb - 2;  // segment: s_bound[seg] <= l < s_bound[seg + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (s_bound[mid] <= l) lo = mid;
            else hi = mid - 1;
        }
        const NodeRec& r = nodes[n - 1 + l];
        for (int k = 0; k < 3; ++k) {
            atomicMin(&s_box[lo][k], float_to_ordered(r.bmin[k]));
            atomicMax(&s_box[lo][3 + k], float_to_ordered(r.bmax[k]));
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int nseg = nb - 1;
    float best = INFINITY;
    uint32_t bk = b + 1;
    for (int i = 1; i < nseg; ++i) {  // candidate s_bound[i]: left = segments 0..i-1
        float llo[3] = {INFINITY, INFINITY, INFINITY}, lhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        float rlo[3] = {INFINITY, INFINITY, INFINITY}, rhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int g = 0; g < nseg; ++g) {
            float* lo3 = g < i ? llo : rlo;
            float* hi3 = g < i ? lhi : rhi;
            for (int k = 0; k < 3; ++k) {
                lo3[k] = fminf(lo3[k], ordered_to_float(s_box[g][k]));
                hi3[k] = fmaxf(hi3[k], ordered_to_float(s_box[g][3 + k]));
            }
        }
        const uint32_t k = s_bound[i];
        const float cst = fadd(saoh_cost(fx, n, b, k, llo, lhi), saoh_cost(fx, n, k, e, rlo, rhi));
        if (cst < best) {  // candidates ascend: the first minimum is the smallest position
            best = cst;
            bk = k;
        }
    }
    const int64_t g = (int64_t)bk - 1;
    int32_t id;
    if (nd.parent < 0) {
        *groot = g;
        id = 0;
    } else {
        const int64_t nm1 = n - 1;
        id = (int32_t)(((g - *groot) % nm1 + nm1) % nm1);
        if (nd.side == 0) left[nd.parent] = id;
        else right[nd.parent] = id;
    }
    parent[id] = nd.parent;
    if (bk - b == 1) {
        left[id] = (int32_t)(n - 1 + b);
        parent[n - 1 + b] = id;
    } else {
        out[atomicAdd(out_count, 1u)] = SaohNode{b, bk, id, 0u};
    }
    if (e - bk == 1) {
        right[id] = (int32_t)(n - 1 + bk);
        parent[n - 1 + bk] = id;
    } else {
        out[atomicAdd(out_count, 1u)] = SaohNode{bk, e, id, 1u};
    }
}

// ---------------------------------------------------------------- median split positions
// Every range [b, e) of at least two lights splits at k = b + floor((e - b) / 2)
// (same light order and id rule as above). Each split position g = k - 1 is
// owned by exactly one internal node: thread g walks down from the root to it
// (at most ceil(log2 n) steps) and writes that node's children and their
// parent links; a child range of one light is its leaf.
__global__ void k_median(int64_t n, int32_t* __restrict__ left, int32_t* __restrict__ right,
                         int32_t* __restrict__ parent)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n - 1) return;
    const int64_t nm1 = n - 1, groot = n / 2 - 1;
    auto id_of = [&](int64_t s) { return (int32_t)(((s - groot) % nm1 + nm1) % nm1); };
    int64_t b = 0, e = n;
    for (int step = 0; step < 64; ++step) {  // g always lies in [b, e - 2]
        const int64_t k = b + (e - b) / 2;
        if (k - 1 == g) {
            const int32_t id = id_of(g);
            const int32_t l = k - b == 1 ? (int32_t)(nm1 + b) : id_of(b + (k - b) / 2 - 1);
            const int32_t r = e - k == 1 ? (int32_t)(nm1 + k) : id_of(k + (e - k) / 2 - 1);
            left[id] = l;
            right[id] = r;
            parent[l] = id;
            parent[r] = id;
            return;
        }
        if (g < k - 1) e = k;
        else b = k;
    }
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int build_tree(rll_ctx* ctx, const float* tri, const float* emission, int64_t n, int builder, rll_tree* t)
{
    cudaStream_t s = ctx->stream;
    const int64_t nn = 2 * n - 1;
    t->n = n;
    cudaError_t e;
#define RLL_ALLOC(ptr, bytes)                                                 \
    e = cudaMalloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 64);               \
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaMalloc(tree)");
    RLL_ALLOC(t->nodes, sizeof(NodeRec) * nn);
    RLL_ALLOC(t->pairs, sizeof(PairRec) * (n - 1));
    RLL_ALLOC(t->quads, sizeof(DescRec) * 4 * (n - 1));
    RLL_ALLOC(t->lights, sizeof(LightRec) * n);
    RLL_ALLOC(t->perm, sizeof(uint32_t) * n);
    RLL_ALLOC(t->left, sizeof(int32_t) * (n - 1));
    RLL_ALLOC(t->right, sizeof(int32_t) * (n - 1));
    RLL_ALLOC(t->parent, sizeof(int32_t) * nn);
    RLL_ALLOC(t->light_cdf, sizeof(float) * n);
#undef RLL_ALLOC
    // scratch: codes, idx, sort, begin/end (unused after build), axis sums,
    // counters, cone minima, bbox, scan sums
    const size_t sort_b = radix_sort_scratch_bytes(n);
    const size_t saoh_b = builder == RLL_TREE_SAOH ? a256(40 * (n + 1)) + 2 * a256(sizeof(SaohNode) * n) + a256(64)
                                                  : 0;
    const size_t need = a256(4 * n) * 2 + sort_b + a256(4 * nn) * 2 + a256(12 * nn) + a256(4 * n) +
                        a256(4 * nn) + a256(64) + a256(4 * 4096) + a256(4 * n) + saoh_b;
    char* w = (char*)ws_get(ctx, need);
    if (!w) return RLL_E_NOMEM;
    uint32_t* codes = (uint32_t*)w; w += a256(4 * n);
    uint32_t* idx = (uint32_t*)w; w += a256(4 * n);
    void* sort_ws = w; w += sort_b;
    uint32_t* begin = (uint32_t*)w; w += a256(4 * nn);
    uint32_t* end = (uint32_t*)w; w += a256(4 * nn);
    float* axis_sum = (float*)w; w += a256(12 * nn);
    uint32_t* counters = (uint32_t*)w; w += a256(4 * n);
    int* cosmin = (int*)w; w += a256(4 * nn);
    int* bbox = (int*)w; w += a256(64);
    void* scan_ws = w; w += a256(4 * 4096);
    float* leaf_phi = (float*)w; w += a256(4 * n);
    long long* fx = (long long*)w; w += builder == RLL_TREE_SAOH ? a256(40 * (n + 1)) : 0;
    SaohNode* list_a = (SaohNode*)w; w += builder == RLL_TREE_SAOH ? a256(sizeof(SaohNode) * n) : 0;
    SaohNode* list_b = (SaohNode*)w; w += builder == RLL_TREE_SAOH ? a256(sizeof(SaohNode) * n) : 0;
    uint32_t* saoh_ctr = (uint32_t*)w;  // [0] next-level count, [2..3] int64 root split, [4..5] max bits

    k_bbox_init<<<1, 32, 0, s>>>(bbox);
    k_centroid_bbox<<<grid_for(n), kBlock, 0, s>>>(tri, n, bbox);
    k_morton<<<grid_for(n), kBlock, 0, s>>>(tri, n, bbox, codes, idx);
    uint32_t *scodes, *sidx;
    e = radix_sort_pairs(s, codes, idx, n, 30, 0xFFFFFFFFu, sort_ws, &scodes, &sidx);
    if (e != cudaSuccess) return check_cuda(ctx, e, "radix sort (tree)");
    e = cudaMemsetAsync(t->parent, 0xFF, sizeof(int32_t) * nn, s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "memset parent");
    if (n > 1 && builder == RLL_TREE_LBVH)
        k_karras<<<grid_for(n - 1), kBlock, 0, s>>>(scodes, sidx, n, t->left, t->right, t->parent, begin, end);
    if (n > 1 && builder == RLL_TREE_MEDIAN) k_median<<<grid_for(n - 1), kBlock, 0, s>>>(n, t->left, t->right, t->parent);
    k_leaves<<<grid_for(n), kBlock, 0, s>>>(tri, emission, n, sidx, t->perm, t->lights, t->nodes, axis_sum);
    if (n > 1 && builder == RLL_TREE_SAOH) {
        int64_t* groot = reinterpret_cast<int64_t*>(saoh_ctr + 2);
        int* mx = reinterpret_cast<int*>(saoh_ctr + 4);
        e = cudaMemsetAsync(saoh_ctr, 0, 64, s);
        if (e != cudaSuccess) return check_cuda(ctx, e, "memset (saoh)");
        k_saoh_max<<<grid_for(n), kBlock, 0, s>>>(n, t->nodes, axis_sum, mx);
        k_saoh_fixed<<<grid_for(n + 1), kBlock, 0, s>>>(n, t->nodes, axis_sum, mx, fx);
        k_saoh_scan<<<5, 1024, 0, s>>>(n, fx);
        const SaohNode root{0u, (uint32_t)n, -1, 0u};
        e = cudaMemcpyAsync(list_a, &root, sizeof(root), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return check_cuda(ctx, e, "saoh root");
        uint32_t count = 1;
        for (int level = 0; count > 0; ++level) {
            if (level > kMaxTreeDepth) return fail(ctx, RLL_E_DEVICE, "saoh build: too many levels");
            e = cudaMemsetAsync(saoh_ctr, 0, sizeof(uint32_t), s);
            if (e != cudaSuccess) return check_cuda(ctx, e, "memset (saoh level)");
            k_saoh_level<<<count, kSaohThreads, 0, s>>>(n, list_a, count, list_b, saoh_ctr, scodes, sidx, t->nodes,
                                                        fx, groot, t->left, t->right, t->parent);
            e = cudaMemcpyAsync(&count, saoh_ctr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return check_cuda(ctx, e, "saoh level");
            SaohNode* tmp = list_a;
            list_a = list_b;
            list_b = tmp;
        }
    }
    e = cudaMemsetAsync(counters, 0, sizeof(uint32_t) * n, s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "memset counters");
    if (n > 1) k_bottom_up<<<grid_for(n), kBlock, 0, s>>>(n, t->left, t->right, t->parent, t->nodes, axis_sum, counters);
    k_axis<<<grid_for(nn), kBlock, 0, s>>>(nn, t->nodes, axis_sum, cosmin);
    k_cone<<<grid_for(n), kBlock, 0, s>>>(n, t->lights, t->nodes, t->parent, cosmin);
    k_finalize<<<grid_for(nn), kBlock, 0, s>>>(nn, t->nodes, cosmin);
    k_pairs<<<grid_for(n), kBlock, 0, s>>>(n, t->nodes, t->left, t->right, t->pairs, leaf_phi);
    if (n > 1) k_quads<<<grid_for(n - 1), kBlock, 0, s>>>(n, t->nodes, t->left, t->right, t->quads);
    e = inclusive_scan_f32(s, leaf_phi, t->light_cdf, n, scan_ws);
    if (e != cudaSuccess) return check_cuda(ctx, e, "scan (light cdf)");
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(ctx, e, "tree kernels");
    // the scratch is reused by later calls: finish before returning
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(ctx, e, "tree build");
    return RLL_OK;
}

int tree_update_emission(rll_ctx* ctx, rll_tree* t, const float* emission)
{
    k_update_emission<<<grid_for(t->n), kBlock, 0, ctx->stream>>>(t->n, t->perm, emission, t->lights);
    return check_cuda(ctx, cudaGetLastError(), "update emission");
}

}  // namespace rll
