// Per-point light sampling shared by the single-grid kernel (sample.cu) and
// the persistent batched kernel (batched.cu): hash lookup / lazy insert, cdf
// binary search, in-cluster choice, light point, shadow test, estimate and
// learning record. See sample.cu for the method notes.
#pragma once

#include <cuda_runtime.h>

#include "learn_core.cuh"  // bitonic_sort_u64
#include "rll_device.cuh"

namespace rll {

// cluster bits of a batched record key (cut sizes up to 64)
constexpr uint32_t kBatchClusterBits = 6;

struct SampleArgs {
    const float* pos;
    const float* nrm;
    const float* albedo;
    int64_t n_points;         // plane stride of pos / nrm / rgb
    int64_t p_begin, p_end;   // points this launch shades (k_sample)
    const float* boxes;
    int n_boxes;
    // the boxes sorted by their lower x bound ([2 n_boxes] float4 (min, max); min.w the running
    // maximum of max.x); nullptr: the boxes as given, all tested
    const float4* boxes_sorted;
    unsigned long long* keys;
    const uint32_t* cut;
    const void* C;
    uint32_t Hl, M, m;        // slots per resolution level, cut size, cut length
    uint32_t levels;          // resolution levels (cell size * 2^l)
    const float* footprint;   // [P] or nullptr (every point at level 0)
    const uint32_t* def_cut;
    const void* def_C;
    float origin[3];
    float h;
    uint32_t nb;
    uint32_t jitter;
    uint32_t reward_mode;
    const PairRec* pairs;
    const DescRec* quads;     // two-level descent records (4 per internal node)
    const NodeRec* nodes;
    const LightRec* lights;
    const float* light_cdf;
    int64_t n_lights;
    unsigned long long seed;
    uint32_t frame;
    int spp;
    float* rgb;
    uint32_t* rec_key;
    float* rec_val;
    int32_t* dbg_light;
    float* dbg_pcut;
    float* dbg_pin;
    uint32_t* status;
    // record key encoding: 0 -> slot * M + cluster (one grid); 1 -> ((cell_base
    // + slot) << kBatchClusterBits) | cluster (many grids sorted together)
    uint32_t key_cells;
    uint32_t cell_base;
};

// Level of a point with footprint f: the smallest l with h * 2^l >= f, i.e.
// ceil(log2(f / h)) from the binary32 quotient (exponent and mantissa bits),
// clamped to [0, levels - 1]; f <= h and NaN give 0.
__device__ __forceinline__ uint32_t footprint_level(float f, float h, uint32_t levels)
{
    const float r = fdiv(f, h);
    if (!(r > 1.0f)) return 0u;
    const uint32_t b = __float_as_uint(r);
    const uint32_t l = ((b >> 23) & 0xFFu) - 127u + ((b & 0x7FFFFFu) != 0u);
    return min(l, levels - 1u);
}

// Lookup with lazy creation in the slot range of one level: linear probing
// from level * Hl + (fmix64(key) mod Hl) for at most kMaxProbes slots.
__device__ __forceinline__ int64_t lookup_insert(unsigned long long* keys, uint32_t Hl, uint32_t level,
                                                 unsigned long long key)
{
    const unsigned long long h = fmix64(key);
    for (int i = 0; i < kMaxProbes; ++i) {
        const uint32_t slot = level * Hl + (uint32_t)((h + (unsigned long long)i) & (unsigned long long)(Hl - 1));
        const unsigned long long k = __ldcg(keys + slot);
        if (k == key) return slot;
        if (k == kEmptyKey) {
            const unsigned long long old = atomicCAS(keys + slot, kEmptyKey, key);
            if (old == kEmptyKey || old == key) return slot;
        }
    }
    return -1;
}

__device__ __forceinline__ DescRec load_desc(const DescRec* p)
{
    DescRec r;
    const float4* s = reinterpret_cast<const float4*>(p);
    float4* d = reinterpret_cast<float4*>(&r);
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = __ldg(s + k);
    return r;
}

__device__ __forceinline__ LightRec load_light(const LightRec* p)
{
    LightRec r;
    const float4* s = reinterpret_cast<const float4*>(p);
    float4* d = reinterpret_cast<float4*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = __ldg(s + k);
    return r;
}

// A shadow segment's direction component: one with |d| < 2^-100 (the segment
// does not move along that axis; 1/d would be infinite and the slab planes
// undefined) is taken as 2^-100 with the sign of d. o * 2^100 is then exact,
// the planes lie at t = (b - o) 2^100 rounded, and the segment is inside that
// slab exactly when b_min < o < b_max -- the decision for a parallel segment.
__device__ __forceinline__ float seg_dir(float d)
{
    return fabsf(d) >= 0x1p-100f ? d : copysignf(0x1p-100f, d);
}

struct ShadeOut {
    float est[3];
    float reward;
};

// light point, shadow test, contribution (x, n: shading point and normal). s_box: the boxes,
// s_box[2b] min and s_box[2b + 1] max; when `sorted`, in increasing order of min.x, with
// s_box[2b].w the largest max.x among boxes 0..b.
__device__ __forceinline__ ShadeOut shade(const LightRec& L, float x0, float x1, float x2, float n0, float n1,
                                          float n2, float albedo, float p_cut, float p_in, float ua, float ub,
                                          const float4* s_box, int n_boxes, uint32_t reward_mode,
                                          bool sorted = false)
{
    const float su = fsqrt(ua);
    const float b0 = fsub(1.0f, su), b1 = fmul(ub, su), b2 = fsub(su, b1);
    const float y0 = fadd(fadd(fmul(b0, L.v0[0]), fmul(b1, L.v1[0])), fmul(b2, L.v2[0]));
    const float y1 = fadd(fadd(fmul(b0, L.v0[1]), fmul(b1, L.v1[1])), fmul(b2, L.v2[1]));
    const float y2 = fadd(fadd(fmul(b0, L.v0[2]), fmul(b1, L.v1[2])), fmul(b2, L.v2[2]));
    const float o0 = fadd(x0, fmul(kShadowOffset, n0));
    const float o1 = fadd(x1, fmul(kShadowOffset, n1));
    const float o2 = fadd(x2, fmul(kShadowOffset, n2));
    const float i0 = fdiv(1.0f, seg_dir(fsub(y0, o0))), i1 = fdiv(1.0f, seg_dir(fsub(y1, o1))),
                i2 = fdiv(1.0f, seg_dir(fsub(y2, o2)));
    const float q0 = -fmul(o0, i0), q1 = -fmul(o1, i1), q2 = -fmul(o2, i2);
    // Conservative prefilter: a box can only block the segment if it meets the
    // segment's bounding box widened by del; del exceeds the rounding error of
    // the slab planes below (a few ulps of |o| + |y|), so no box the exact
    // slab test would report is skipped and the decision is unchanged.
    const float e0 = 1e-5f * (1.0f + fabsf(o0) + fabsf(y0));
    const float e1 = 1e-5f * (1.0f + fabsf(o1) + fabsf(y1));
    const float e2 = 1e-5f * (1.0f + fabsf(o2) + fabsf(y2));
    const float lo0 = fminf(o0, y0) - e0, hi0 = fmaxf(o0, y0) + e0;
    const float lo1 = fminf(o1, y1) - e1, hi1 = fmaxf(o1, y1) + e1;
    const float lo2 = fminf(o2, y2) - e2, hi2 = fmaxf(o2, y2) + e2;
    // With the boxes sorted by min.x, the boxes before the first one whose running maximum of max.x
    // reaches lo0 all have max.x < lo0, and those from the first one with min.x > hi0 on all have
    // min.x > hi0: the prefilter below rejects every box outside that run, so testing the run
    // alone gives the decision of the full loop.
    int b = 0;
    const int b_end = n_boxes;
    if (sorted) {
        int lo = 0, hi = n_boxes;  // first box whose running maximum of max.x is >= lo0
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_box[2 * mid].w < lo0) lo = mid + 1;
            else hi = mid;
        }
        b = lo;
    }
    bool occluded = false;
    for (; b < b_end && !occluded; ++b) {
        const float4 bmin = s_box[2 * b], bmax = s_box[2 * b + 1];
        if (sorted && bmin.x > hi0) break;
        if (bmin.x > hi0 || bmax.x < lo0 || bmin.y > hi1 || bmax.y < lo1 || bmin.z > hi2 || bmax.z < lo2) continue;
        const float ta0 = __fmaf_rn(bmin.x, i0, q0), tb0 = __fmaf_rn(bmax.x, i0, q0);
        const float ta1 = __fmaf_rn(bmin.y, i1, q1), tb1 = __fmaf_rn(bmax.y, i1, q1);
        const float ta2 = __fmaf_rn(bmin.z, i2, q2), tb2 = __fmaf_rn(bmax.z, i2, q2);
        float tn = fmaxf(0.0f, fminf(ta0, tb0));
        float tf = fminf(kShadowTmax, fmaxf(ta0, tb0));
        tn = fmaxf(tn, fminf(ta1, tb1));
        tf = fminf(tf, fmaxf(ta1, tb1));
        tn = fmaxf(tn, fminf(ta2, tb2));
        tf = fminf(tf, fmaxf(ta2, tb2));
        occluded = tn < tf;
    }
    ShadeOut o;
    const float wx = y0 - x0, wy = y1 - x1, wz = y2 - x2;
    const float d2 = wx * wx + wy * wy + wz * wz;
    const float inv_d = rsqrtf(d2);
    const float cx = fmaxf(0.0f, (n0 * wx + n1 * wy + n2 * wz) * inv_d);
    const float cl = fmaxf(0.0f, -(L.n[0] * wx + L.n[1] * wy + L.n[2] * wz) * inv_d);
    const float geo = (occluded || !(d2 > 0.0f)) ? 0.0f : __fdividef(cx * cl, d2);
    const float f = albedo * 0.31830988618379067f;
    const float c0 = f * L.le[0] * geo, c1 = f * L.le[1] * geo, c2 = f * L.le[2] * geo;
    // a zero contribution is zero whatever its pdf (a long-unrewarded
    // cluster's probability may underflow binary32)
    const float w = geo > 0.0f ? __fdividef(__fdividef(L.area, p_cut), p_in) : 0.0f;
    o.est[0] = c0 * w;
    o.est[1] = c1 * w;
    o.est[2] = c2 * w;
    const float lum = 0.2126f * c0 + 0.7152f * c1 + 0.0722f * c2;
    o.reward = !(lum > 0.0f) ? 0.0f : (reward_mode == RLL_REWARD_CLUSTER ? __fdividef(lum * L.area, p_in) : lum * L.area);
    return o;
}

// MINB: resident blocks per SM the register allocation is held to (3: no
// cap at 256 threads, 4: at most 64 registers per thread).
// Boxes in shared memory as float4 pairs: s_box[2b] = (min xyz, 0),
// s_box[2b + 1] = (max xyz, 0). Filled by all threads of the block.
__device__ __forceinline__ void stage_boxes(float4* s_box, const float* boxes, int n_boxes)
{
    for (int b = threadIdx.x; b < n_boxes; b += blockDim.x) {
        const float* bx = boxes + 6 * b;
        s_box[2 * b] = make_float4(bx[0], bx[1], bx[2], 0.0f);
        s_box[2 * b + 1] = make_float4(bx[3], bx[4], bx[5], 0.0f);
    }
}

// The occluder boxes sorted by their lower x bound (ties by index) for the shadow test's early
// start and stop, by the whole block: a bitonic network over (ordered min.x << 32 | index) keys in
// shared memory. Output: [2 n] float4 (min, max) in that order, the min's w holding the running
// maximum of max.x over the boxes up to this one (nondecreasing). n <= kMaxBoxes.
struct SortBoxBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

__device__ __forceinline__ void sort_boxes_block(const float* __restrict__ boxes, int n, float4* __restrict__ out)
{
    __shared__ unsigned long long s_key[kMaxBoxes];
    __shared__ float s_hx[kMaxBoxes];  // max.x in sorted order, then its running maximum
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        s_key[b] = ((unsigned long long)(uint32_t)(float_to_ordered(boxes[6 * b]) ^ (int)0x80000000) << 32) |
                   (uint32_t)b;
    __syncthreads();
    bitonic_sort_u64(s_key, (uint32_t)n, threadIdx.x, blockDim.x, SortBoxBarrier{});
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_hx[i] = boxes[6 * (uint32_t)s_key[i] + 3];
    __syncthreads();
    if (threadIdx.x < 32) {  // running maximum: each lane scans a run, the lanes combine by shuffles
        const int lane = threadIdx.x, per = (n + 31) / 32, b0 = lane * per, b1 = min(n, b0 + per);
        float m = -INFINITY;
        for (int i = b0; i < b1; ++i) m = fmaxf(m, s_hx[i]);
        float incl = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = fmaxf(incl, y);
        }
        float run = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) run = -INFINITY;
        for (int i = b0; i < b1; ++i) {
            run = fmaxf(run, s_hx[i]);
            s_hx[i] = run;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float* bx = boxes + 6 * (uint32_t)s_key[i];
        out[2 * i] = make_float4(bx[0], bx[1], bx[2], s_hx[i]);
        out[2 * i + 1] = make_float4(bx[3], bx[4], bx[5], 0.0f);
    }
}

// The boxes as sorted by sort_boxes_block (2 n_boxes float4), copied as they are.
__device__ __forceinline__ void stage_sorted_boxes(float4* s_box, const float4* sorted, int n_boxes)
{
    for (int i = threadIdx.x; i < 2 * n_boxes; i += blockDim.x) s_box[i] = sorted[i];
}

// Cell, cluster and triangle draws of one sample (draws 0-2 and 4-8).
struct Setup {
    uint32_t node;   // cut node of the chosen cluster
    float p_cut;     // its probability under the cell's cdf
    float ua, ub;    // triangle point draws
    uint32_t rec;    // learning record key (kInvalidRecord if the table is full)
    int64_t slot;
    uint32_t s;
};

template <int P>
__device__ __forceinline__ Setup setup_sample(const SampleArgs& a, SampleStream& rs, float x0, float x1, float x2,
                                              float n0, float n1, float n2, uint32_t level)
{
    using T = typename Store<P>::T;
    const T* Ctab = static_cast<const T*>(a.C);
    const T* Cdef = static_cast<const T*>(a.def_C);
    const uint32_t m = a.m;
    float jit[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (a.jitter) {
#pragma unroll
        for (int k = 0; k < 5; ++k) jit[k] = rs.draw(kDrawJit + k);
    }
    const float h_cell = fmul(a.h, (float)(1u << level));  // exact: a power of two
    const unsigned long long key = cell_key(x0, x1, x2, n0, n1, n2, a.origin, h_cell, a.nb, a.jitter != 0, jit);
    const int64_t slot = lookup_insert(a.keys, a.Hl, level, key);
    const T* crow;
    const uint32_t* cutrow;
    if (slot >= 0) {
        crow = Ctab + slot * a.M;
        cutrow = a.cut + slot * a.M;
    } else {
        crow = Cdef;
        cutrow = a.def_cut;
        atomicOr(a.status, (uint32_t)RLL_E_TABLE_FULL);
    }
    // cluster: first s with C(s) > u * C(m-1)
    const float u = rs.draw(kDrawCut);
    const float total = Store<P>::load(crow[m - 1]);
    uint32_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__fmaf_rn(-u, total, Store<P>::load(crow[mid])) > 0.0f) hi = mid;
        else lo = mid + 1;
    }
    Setup o;
    o.s = lo;
    o.slot = slot;
    const float cprev = lo > 0 ? Store<P>::load(crow[lo - 1]) : 0.0f;
    o.p_cut = (Store<P>::load(crow[lo]) - cprev) / total;
    o.node = cutrow[lo];
    if ((int64_t)o.node >= 2 * a.n_lights - 1) {  // corrupt cut row: flag, sample from the root
        atomicOr(a.status, (uint32_t)RLL_E_DEVICE);
        o.node = 0;
    }
    o.ua = rs.draw(kDrawTriA);
    o.ub = rs.draw(kDrawTriB);
    o.rec = slot < 0 ? kInvalidRecord
                     : (a.key_cells ? ((a.cell_base + (uint32_t)slot) << kBatchClusterBits) | lo
                                    : (uint32_t)slot * a.M + lo);
    return o;
}

// One level of the bound-driven descent below internal node `node` (ud: the
// level's draw; x*: the shading point, n*: its normal broadcast to both
// components). Both children's bounds in one packed evaluation; they are
// compared without a division: w_L = num_L den_R, w_R = num_R den_L; their
// powers if both vanish.
__device__ __forceinline__ void descent_step(const SampleArgs& a, uint32_t& node, float& p_in, float ud,
                                             float x0, float x1, float x2, float2 n0, float2 n1, float2 n2)
{
    PairRec q;
    {
        const float4* src = reinterpret_cast<const float4*>(a.pairs + node);
        float4* dst = reinterpret_cast<float4*>(&q);
#pragma unroll
        for (int k = 0; k < 5; ++k) dst[k] = __ldg(src + k);
    }
    const Bound2 b = importance2(q, x0, x1, x2, n0, n1, n2);
    const float2 w = __fmul2_rn(b.num, make_float2(b.den.y, b.den.x));
    float wl = w.x, wr = w.y;
    float ssum = fadd(wl, wr);
    if (!(ssum > 0.0f)) {
        wl = q.phi.x;
        wr = q.phi.y;
        ssum = fadd(wl, wr);
    }
    bool left;
    float ratio;
    if (ssum > 0.0f) {
        left = __fmaf_rn(ud, ssum, -wl) < 0.0f;
        ratio = __fdividef(left ? wl : wr, wl + wr);  // continuous: pdf only
    } else {
        left = ud < 0.5f;
        ratio = 0.5f;
    }
    p_in *= ratio;
    node = left ? q.id.x : q.id.y;
}

__device__ __forceinline__ void prefetch_l1(const void* p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// One step of the two-level descent below internal node `node` (ud: the
// step's draw): candidates quads[4 node ..] (2 to 4 valid, in light order),
// weights num / max(den, 1e-30), binary32 prefix sums in order; the first
// prefix above u * S is chosen (exact, one fma), probability (P_i -
// P_{i-1}) / S; powers, then uniform over the valid candidates, when all
// weights vanish. Candidates 2 and 3 are prefetched into L1 while 0 and 1
// are evaluated, so no registers hold them meanwhile.
__device__ __forceinline__ void descent2_step(const SampleArgs& a, uint32_t& node, float& p_in, float ud, float x0,
                                              float x1, float x2, float n0, float n1, float n2)
{
    const DescRec* q = a.quads + 4 * (int64_t)node;
    prefetch_l1(q + 2);
    prefetch_l1(reinterpret_cast<const char*>(q + 2) + 64);
    float w[4];
    bool valid3 = false, valid4 = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const DescRec A = load_desc(q + 2 * h), B = load_desc(q + 2 * h + 1);
        const Bound ba = importance(A, x0, x1, x2, n0, n1, n2);
        const Bound bb = importance(B, x0, x1, x2, n0, n1, n2);
        w[2 * h] = fdiv(ba.num, fmaxf(ba.den, 1e-30f));
        w[2 * h + 1] = fdiv(bb.num, fmaxf(bb.den, 1e-30f));
        if (h == 1) {
            valid3 = A.id != 0xFFFFFFFFu;
            valid4 = B.id != 0xFFFFFFFFu;
        }
    }
    const int k = 2 + valid3 + valid4;  // valid candidates come first
    float pre[4], S = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        S = fadd(S, i < k ? w[i] : 0.0f);
        pre[i] = S;
    }
    if (!(S > 0.0f)) {  // rare: the candidates' powers (read again, L1)
        S = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            S = fadd(S, i < k ? __ldg(&q[i].phi) : 0.0f);
            pre[i] = S;
        }
    }
    int pick;
    if (S > 0.0f) {
        pick = k - 1;
#pragma unroll
        for (int i = 3; i >= 0; --i)
            if (i < k && __fmaf_rn(ud, S, -pre[i]) < 0.0f) pick = i;
    } else {
        const uint32_t u24v = (uint32_t)(ud * 16777216.0f);
        pick = (int)(((unsigned long long)u24v * (unsigned long long)k) >> 24);
    }
    // the chosen candidate's interval by selects (no indexed arrays), its id from L1
    float lo = 0.0f, hi = pre[0];
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        if (pick == i) {
            lo = pre[i - 1];
            hi = pre[i];
        }
    }
    p_in *= S > 0.0f ? (hi - lo) / S : 1.0f / (float)k;  // continuous: pdf only
    node = __ldg(&q[pick].id);
}

// Light index of the node a descent ended on. A descent that ran into the
// depth bound (only on a corrupt tree: no builder comes near it) is flagged
// and takes the first light of the node it reached.
__device__ __forceinline__ int64_t leaf_or_flag(const SampleArgs& a, uint32_t node, int64_t nl1)
{
    if ((int64_t)node >= nl1) return (int64_t)node - nl1;
    atomicOr(a.status, (uint32_t)RLL_E_DEVICE);
    return (int64_t)a.nodes[node].begin;
}

// All samples of shading point p, one thread (s_box: see stage_boxes).
template <int P, int MODE, bool DBG>
__device__ __forceinline__ void sample_point(const SampleArgs& a, int64_t p, const float4* s_box)
{
    const int64_t np = a.n_points;
    const float x0 = a.pos[p], x1 = a.pos[np + p], x2 = a.pos[2 * np + p];
    const float n0 = a.nrm[p], n1 = a.nrm[np + p], n2 = a.nrm[2 * np + p];
    const float alb = a.albedo[p];
    const uint32_t level = a.footprint ? footprint_level(__ldg(a.footprint + p), a.h, a.levels) : 0u;
    const int64_t nl1 = a.n_lights - 1;
    const uint32_t nl1u = (uint32_t)nl1;  // internal node ids are below it (at most 2^24 lights)
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;
    for (int j = 0; j < a.spp; ++j) {
        const uint32_t sid = (uint32_t)(p * a.spp + j);
        SampleStream rs;
        rs.init(a.seed, sid, a.frame);
        const Setup su = setup_sample<P>(a, rs, x0, x1, x2, n0, n1, n2, level);
        uint32_t node = su.node;
        float p_in = 1.0f;
        int64_t light;
        if (MODE == RLL_MODE_UNIFORM) {
            const NodeRec& r = a.nodes[node];
            const uint32_t w = r.end - r.begin;
            const uint32_t u24v = (uint32_t)(rs.draw(kDrawUniform) * 16777216.0f);
            light = (int64_t)r.begin + (int64_t)(((unsigned long long)u24v * w) >> 24);
            p_in = 1.0f / (float)w;
        } else if (MODE == RLL_MODE_DESCENT2) {
            for (uint32_t level = 0; node < nl1u && level < (uint32_t)kMaxTreeDepth; ++level)
                descent2_step(a, node, p_in, rs.draw(kDrawDescent + level), x0, x1, x2, n0, n1, n2);
            light = leaf_or_flag(a, node, nl1);
        } else {
            const float2 vn0 = make_float2(n0, n0), vn1 = make_float2(n1, n1), vn2 = make_float2(n2, n2);
            // level l takes draw kDrawDescent + l: words 1..3 of Philox block 2, then four levels per
            // block, unrolled so that every word index is a constant
            static_assert(kDrawDescent == 9, "descent draws start at word 1 of block 2");
            uint4 w = rs.block_words(2);
            if (node < nl1u) descent_step(a, node, p_in, u24(w.y), x0, x1, x2, vn0, vn1, vn2);
            if (node < nl1u) descent_step(a, node, p_in, u24(w.z), x0, x1, x2, vn0, vn1, vn2);
            if (node < nl1u) descent_step(a, node, p_in, u24(w.w), x0, x1, x2, vn0, vn1, vn2);
            for (uint32_t b = 3; node < nl1u && b < (uint32_t)(kMaxTreeDepth / 4); ++b) {
                w = rs.block_words(b);
                descent_step(a, node, p_in, u24(w.x), x0, x1, x2, vn0, vn1, vn2);
                if (node < nl1u) descent_step(a, node, p_in, u24(w.y), x0, x1, x2, vn0, vn1, vn2);
                if (node < nl1u) descent_step(a, node, p_in, u24(w.z), x0, x1, x2, vn0, vn1, vn2);
                if (node < nl1u) descent_step(a, node, p_in, u24(w.w), x0, x1, x2, vn0, vn1, vn2);
            }
            light = leaf_or_flag(a, node, nl1);
        }
        const LightRec Lr = load_light(a.lights + light);
        const ShadeOut o = shade(Lr, x0, x1, x2, n0, n1, n2, alb, su.p_cut, p_in, su.ua, su.ub, s_box, a.n_boxes,
                                 a.reward_mode, a.boxes_sorted != nullptr);
        acc0 += o.est[0];
        acc1 += o.est[1];
        acc2 += o.est[2];
        if (a.rec_key) {
            a.rec_key[sid] = su.rec;
            a.rec_val[sid] = o.reward;
        }
        if (DBG) {
            if (a.dbg_light) a.dbg_light[sid] = (int32_t)light;
            if (a.dbg_pcut) a.dbg_pcut[sid] = su.p_cut;
            if (a.dbg_pin) a.dbg_pin[sid] = p_in;
        }
    }
    const float inv_spp = 1.0f / (float)a.spp;
    a.rgb[p] = acc0 * inv_spp;
    a.rgb[np + p] = acc1 * inv_spp;
    a.rgb[2 * np + p] = acc2 * inv_spp;
}

}  // namespace rll
