// Device-side building blocks of the GB300 Reinforcement Lightcuts Learning
// library: record layouts, Philox4x32-10, the binary32 decision arithmetic,
// table storage formats.
//
// Decision arithmetic. Every floating-point value that decides an integer
// (hash cell, Morton code, descent branch, shadow test, split choice) is
// evaluated with explicitly rounded binary32 intrinsics (__fadd_rn, __fmul_rn,
// ...), so that no multiply-add is contracted and the result is the IEEE
// value of the stated formula. Continuous quantities (contribution, pdf,
// reward) use ordinary fp32 arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/rll.h"

namespace rll {

constexpr unsigned long long kEmptyKey = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t kInvalidRecord = 0xFFFFFFFFu;
constexpr int kMaxProbes = 64;
constexpr int kMaxCut = 256;
// Bound of every walk over the light tree: far above any builder's depth (radix tree of 64-bit
// keys: <= 64 levels; SAOH: < 250 levels at 2^24 lights; median: ceil(log2 n)).
constexpr int kMaxTreeDepth = 4096;
constexpr int kMaxBoxes = 1024;
constexpr uint32_t kMaxSplitIterations = 256;
constexpr float kShadowOffset = 1e-4f;
constexpr float kShadowTmax = 0.9999f;

// Node bounds record, 64 bytes (every node: export, uniform in-cluster
// choice, split-collapse).
struct __align__(16) NodeRec {
    float bmin[3];
    float bmax[3];
    float phi;       // power bound: sum over lights of lum(Le) * area
    float axis[3];   // orientation cone axis
    float cos_t;     // orientation cone: cos of the half angle
    uint32_t id;     // node id (leaf of sorted light l: n - 1 + l)
    uint32_t begin;  // first sorted light
    uint32_t end;    // one past the last sorted light
};
static_assert(sizeof(NodeRec) == 64, "NodeRec must be 64 bytes");

// Descent record of one child, 48 bytes: the constants of the importance
// bound precomputed (binary32, same operations as on the fly). The two-level
// descent reads them four per internal node (quads).
struct __align__(16) DescRec {
    float c[3];      // AABB centre
    float r2;        // squared half diagonal
    float r;         // half diagonal
    float phi;       // power bound
    float axis[3];   // cone axis
    float cos_t;     // cone cos(theta)
    float sin_t;     // cone sin(theta)
    uint32_t id;     // node id
};
static_assert(sizeof(DescRec) == 48, "DescRec must be 48 bytes");

// The DescRec fields of both children of one internal node, interleaved
// (x: left child, y: right child) so that each 16-byte load yields two packed
// operands of the paired bound below; 80 bytes per descent level (the
// descent is bound by how many record bytes a level pulls through L1). r2 is
// r r, formed at use; cs holds (1 - cos theta, sin theta) of each child as two
// binary16 values (exactly the DescRec values; cos theta = 1 - v is exact).
struct __align__(16) PairRec {
    float2 c0, c1, c2, r, phi;
    float2 a0, a1, a2;
    uint2 cs;
    uint2 id;
};
static_assert(sizeof(PairRec) == 80, "PairRec must be 80 bytes");

// Sorted light, 64 bytes.
struct __align__(16) LightRec {
    float v0[3];
    float v1[3];
    float v2[3];
    float le[3];     // current RGB radiance
    float n[3];      // unit winding normal
    float area;
};
static_assert(sizeof(LightRec) == 64, "LightRec must be 64 bytes");

// ---------------------------------------------------------------- exact ops
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, key bumped by 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// uniform in [0, 1): top 24 bits times 2^-24 (exact in binary32)
__device__ __forceinline__ float u24(uint32_t x) { return __uint2float_rn(x >> 8) * 0x1p-24f; }

// Draw layout of one light sample: draw i is word (i mod 4) of
// Philox(counter = (sample id, frame, i / 4, 0), key = (seed lo, seed hi)).
//   0 cut search, 1-2 triangle point, 3 uniform in-cluster choice,
//   4-7 jitter x, y, z, normal u, 8 jitter normal v, 9 + k descent level k.
enum : uint32_t {
    kDrawCut = 0, kDrawTriA = 1, kDrawTriB = 2, kDrawUniform = 3, kDrawJit = 4, kDrawDescent = 9
};

struct SampleStream {
    uint2 key;
    uint32_t sample_id, frame;
    uint32_t block;
    uint4 words;

    __device__ __forceinline__ void init(unsigned long long seed, uint32_t sid, uint32_t fr)
    {
        key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
        sample_id = sid;
        frame = fr;
        block = 0xFFFFFFFFu;
    }
    // the four words of Philox block b (draws 4b .. 4b + 3)
    __device__ __forceinline__ uint4 block_words(uint32_t b)
    {
        if (b != block) {
            words = philox4x32_10(make_uint4(sample_id, frame, b, 0u), key);
            block = b;
        }
        return words;
    }
    __device__ __forceinline__ float draw(uint32_t i)
    {
        const uint32_t b = i >> 2;
        if (b != block) {
            words = philox4x32_10(make_uint4(sample_id, frame, b, 0u), key);
            block = b;
        }
        const uint32_t k = i & 3u;
        const uint32_t w = k == 0 ? words.x : (k == 1 ? words.y : (k == 2 ? words.z : words.w));
        return u24(w);
    }
};

// ---------------------------------------------------------------- hashing
// MurmurHash3 64-bit finaliser (Appleby).
__device__ __forceinline__ unsigned long long fmix64(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__device__ __forceinline__ uint32_t quant_pos(float p, float o, float h, bool jit, float u)
{
    float t = fdiv(fsub(p, o), h);
    if (jit) t = fadd(t, fsub(u, 0.5f));
    float f = floorf(t);
    f = fminf(fmaxf(f, -32767.0f), 32766.0f);
    return (uint32_t)((int)f + 32768);
}

__device__ __forceinline__ uint32_t quant_nrm(float a, uint32_t nb, bool jit, float u)
{
    float q = fmul(fmul(fadd(a, 1.0f), 0.5f), (float)nb);
    if (jit) q = fadd(q, fsub(u, 0.5f));
    float f = floorf(q);
    f = fminf(fmaxf(f, 0.0f), (float)(nb - 1));
    return (uint32_t)f;
}

// 5-d cell key: 16-bit biased x, y, z cells, 8-bit octahedral normal bins
// (y up). Never equals kEmptyKey (the top byte is at most 254).
__device__ __forceinline__ unsigned long long cell_key(float px, float py, float pz, float nx, float ny,
                                                       float nz, const float origin[3], float h,
                                                       uint32_t nb, bool jit, const float j[5])
{
    const uint32_t fx = quant_pos(px, origin[0], h, jit, j[0]);
    const uint32_t fy = quant_pos(py, origin[1], h, jit, j[1]);
    const uint32_t fz = quant_pos(pz, origin[2], h, jit, j[2]);
    const float s = fadd(fadd(fabsf(nx), fabsf(ny)), fabsf(nz));
    float a = 0.0f, b = 0.0f;
    if (s > 0.0f) {
        a = fdiv(nx, s);
        b = fdiv(nz, s);
        if (ny < 0.0f) {
            const float sa = a >= 0.0f ? 1.0f : -1.0f, sb = b >= 0.0f ? 1.0f : -1.0f;
            const float na = fmul(fsub(1.0f, fabsf(b)), sa);
            const float nbv = fmul(fsub(1.0f, fabsf(a)), sb);
            a = na;
            b = nbv;
        }
    }
    const uint32_t iu = quant_nrm(a, nb, jit, j[3]);
    const uint32_t iv = quant_nrm(b, nb, jit, j[4]);
    return (unsigned long long)fx | ((unsigned long long)fy << 16) | ((unsigned long long)fz << 32) |
           ((unsigned long long)iu << 48) | ((unsigned long long)iv << 56);
}

// ---------------------------------------------------------------- bounds
// Descent constants of a node (centre, r^2, r, sin theta).
__device__ __forceinline__ DescRec make_desc(const NodeRec& n)
{
    DescRec d;
    const float ex = fsub(n.bmax[0], n.bmin[0]), ey = fsub(n.bmax[1], n.bmin[1]), ez = fsub(n.bmax[2], n.bmin[2]);
    for (int k = 0; k < 3; ++k) {
        d.c[k] = fmul(fadd(n.bmin[k], n.bmax[k]), 0.5f);
        d.axis[k] = n.axis[k];
    }
    // compact constants: r rounded up one ulp and r^2 = r r (not below the box's squared half
    // diagonal); the cone as v = 1 - cos theta rounded up to binary16 (a cone at least as wide;
    // 11 significant bits of v keep narrow cones narrow), cos = 1 - v (exact), and sin theta of
    // that cone rounded up to binary16 from the exact 1 - cos^2 = v (2 - v). Rounding up twice
    // (binary32, then binary16) equals rounding up once.
    const float rb2 = fmul(0.25f, fadd(fadd(fmul(ex, ex), fmul(ey, ey)), fmul(ez, ez)));
    d.r = nextafterf(fsqrt(rb2), INFINITY);
    d.r2 = fmul(d.r, d.r);
    d.phi = n.phi;
    const float v = __half2float(__float2half_ru(__fsub_ru(1.0f, n.cos_t)));
    d.cos_t = fsub(1.0f, v);
    d.sin_t = __half2float(__float2half_ru(__fsqrt_ru(fmul(v, fsub(2.0f, v)))));
    d.id = n.id;
    return d;
}

// Unoccluded importance of a node seen from (x, n): power times the receiver
// and emitter cosine bounds over the node's bounding sphere, over distance^2,
// kept as num / den = (phi A B) / d^6 with A = d^2 Brecv, B = d^2 Bemit.
// Cosines and sines are carried multiplied by |d| (2-3 square roots, no
// division).
struct Bound {
    float num, den;
};

__device__ __forceinline__ Bound importance(const DescRec& r, float x0, float x1, float x2, float n0, float n1,
                                            float n2)
{
    const float dx = fsub(r.c[0], x0), dy = fsub(r.c[1], x1), dz = fsub(r.c[2], x2);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, fmul(dx, dx)));
    if (d2 <= r.r2) return Bound{r.phi, fmaxf(r.r2, 1e-30f)};
    const float cb = fsqrt(fsub(d2, r.r2));
    const float nd = __fmaf_rn(n2, dz, __fmaf_rn(n1, dy, fmul(n0, dx)));
    float A = d2;
    if (nd < cb) A = fmaxf(0.0f, __fmaf_rn(nd, cb, fmul(fsqrt(fmaxf(0.0f, __fmaf_rn(-nd, nd, d2))), r.r)));
    const float ad = -__fmaf_rn(r.axis[2], dz, __fmaf_rn(r.axis[1], dy, fmul(r.axis[0], dx)));
    const float sphi = __fmaf_rn(r.sin_t, cb, fmul(r.cos_t, r.r));
    const float cphi = __fmaf_rn(r.cos_t, cb, -fmul(r.sin_t, r.r));
    float B = d2;
    if (!(sphi <= 0.0f || cphi <= ad))
        B = fmaxf(0.0f, __fmaf_rn(ad, cphi, fmul(fsqrt(fmaxf(0.0f, __fmaf_rn(-ad, ad, d2))), sphi)));
    return Bound{fmul(fmul(r.phi, A), B), fmul(fmul(d2, d2), d2)};
}

// importance() of both children of a node at once, in packed binary32
// (f32x2) arithmetic: per component the same correctly rounded operations in
// the same order as importance(), hence bit-identical bounds. d2 - r2 is
// computed as d2 + (-r2) and d2 <= r2 as d2 - r2 <= 0 (equal under round to
// nearest with gradual underflow); the early return inside the bounding
// sphere becomes a per-component select. The receiver and emitter branches
// are evaluated for both components always and selected per component (in a
// warp some lane nearly always needs them, so the branches only cost their
// divergence; the values selected are the same). n*: the normal broadcast to
// both components.
struct Bound2 {
    float2 num, den;
};

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

__device__ __forceinline__ Bound2 importance2(const PairRec& q, float x0, float x1, float x2, float2 n0, float2 n1,
                                              float2 n2)
{
    const float2 nr2 = neg2(__fmul2_rn(q.r, q.r));
    const float2 cl = __half22float2(*reinterpret_cast<const __half2*>(&q.cs.x));
    const float2 cr = __half22float2(*reinterpret_cast<const __half2*>(&q.cs.y));
    const float2 cos_t = __fadd2_rn(make_float2(1.0f, 1.0f), neg2(make_float2(cl.x, cr.x)));  // exact
    const float2 sin_t = make_float2(cl.y, cr.y);
    const float2 dx = make_float2(fsub(q.c0.x, x0), fsub(q.c0.y, x0));
    const float2 dy = make_float2(fsub(q.c1.x, x1), fsub(q.c1.y, x1));
    const float2 dz = make_float2(fsub(q.c2.x, x2), fsub(q.c2.y, x2));
    const float2 d2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const float2 t = __fadd2_rn(d2, nr2);
    const bool in_x = t.x <= 0.0f, in_y = t.y <= 0.0f;
    const float2 cb = make_float2(fsqrt(t.x), fsqrt(t.y));
    const float2 nd = __ffma2_rn(n2, dz, __ffma2_rn(n1, dy, __fmul2_rn(n0, dx)));
    float2 A = d2;
    const bool ra = nd.x < cb.x, rb = nd.y < cb.y;
    {
        const float2 g = __ffma2_rn(neg2(nd), nd, d2);
        const float2 sq = make_float2(fsqrt(fmaxf(0.0f, g.x)), fsqrt(fmaxf(0.0f, g.y)));
        const float2 v = __ffma2_rn(nd, cb, __fmul2_rn(sq, q.r));
        A.x = ra ? fmaxf(0.0f, v.x) : A.x;
        A.y = rb ? fmaxf(0.0f, v.y) : A.y;
    }
    const float2 ad = neg2(__ffma2_rn(q.a2, dz, __ffma2_rn(q.a1, dy, __fmul2_rn(q.a0, dx))));
    const float2 sphi = __ffma2_rn(sin_t, cb, __fmul2_rn(cos_t, q.r));
    const float2 cphi = __ffma2_rn(cos_t, cb, neg2(__fmul2_rn(sin_t, q.r)));
    float2 B = d2;
    const bool ea = !(sphi.x <= 0.0f || cphi.x <= ad.x), eb = !(sphi.y <= 0.0f || cphi.y <= ad.y);
    {
        const float2 g = __ffma2_rn(neg2(ad), ad, d2);
        const float2 sq = make_float2(fsqrt(fmaxf(0.0f, g.x)), fsqrt(fmaxf(0.0f, g.y)));
        const float2 v = __ffma2_rn(ad, cphi, __fmul2_rn(sq, sphi));
        B.x = ea ? fmaxf(0.0f, v.x) : B.x;
        B.y = eb ? fmaxf(0.0f, v.y) : B.y;
    }
    Bound2 o;
    o.num = __fmul2_rn(__fmul2_rn(q.phi, A), B);
    o.den = __fmul2_rn(__fmul2_rn(d2, d2), d2);
    if (in_x) {
        o.num.x = q.phi.x;
        o.den.x = fmaxf(-nr2.x, 1e-30f);
    }
    if (in_y) {
        o.num.y = q.phi.y;
        o.den.y = fmaxf(-nr2.y, 1e-30f);
    }
    return o;
}

// ---------------------------------------------------------------- storage
template <int P> struct Store;
template <> struct Store<RLL_PREC_FP32> {
    using T = float;
    __device__ __forceinline__ static float load(T v) { return v; }
    __device__ __forceinline__ static T store(float v) { return v; }
    __device__ __forceinline__ static uint16_t bits(T) { return 0; }
};
template <> struct Store<RLL_PREC_FP16> {
    using T = __half;
    __device__ __forceinline__ static float load(T v) { return __half2float(v); }
    // saturating: values beyond the largest finite half are stored as 65504
    __device__ __forceinline__ static T store(float v)
    {
        return __float2half_rn(fminf(fmaxf(v, -65504.0f), 65504.0f));
    }
    __device__ __forceinline__ static uint16_t bits(T v) { return __half_as_ushort(v); }
    __device__ __forceinline__ static T from_bits(uint16_t b) { return __ushort_as_half(b); }
};
template <> struct Store<RLL_PREC_BF16> {
    using T = __nv_bfloat16;
    __device__ __forceinline__ static float load(T v) { return __bfloat162float(v); }
    __device__ __forceinline__ static T store(float v)
    {
        const float mx = 3.3895313892515355e38f;  // largest finite bfloat16
        return __float2bfloat16_rn(fminf(fmaxf(v, -mx), mx));
    }
    __device__ __forceinline__ static uint16_t bits(T v) { return __bfloat16_as_ushort(v); }
    __device__ __forceinline__ static T from_bits(uint16_t b) { return __ushort_as_bfloat16(b); }
};

// Programmatic dependent launch: a kernel launched by launch_pdl may be
// scheduled while the kernel before it on the stream is finishing; its first
// statement is pdl_begin(): wait until that kernel (and so all earlier work)
// has completed and its writes are visible, then let the next kernel be
// scheduled in turn.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ordered-integer image of a float for atomicMin / atomicMax
__device__ __forceinline__ int float_to_ordered(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float ordered_to_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace rll
