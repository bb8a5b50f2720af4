// Per-cell learning and split-collapse shared by the single-grid kernels
// (learn.cu) and the batched kernels (batched.cu). One warp works on one
// cell; q, c, cs, nc, bits are that warp's shared-memory rows (kMaxCut each).
#pragma once

#include <cuda_runtime.h>

#include <climits>

#include "rll_device.cuh"

namespace rll {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Eq. 2 with the floor: q holds the stored Q of one row (m values, shared
// memory); c and bits are shared scratch of the same length. Writes the
// stored cdf row. Called by all 32 lanes of a warp.
template <int P>
__device__ void warp_rebuild_cdf(const float* q, int m, float eps, typename Store<P>::T* out, float* c,
                                 uint16_t* bits)
{
    const int lane = threadIdx.x & 31;
    float part = 0.0f, qmax = 0.0f;
    for (int s = lane; s < m; s += 32) {
        part += q[s];
        qmax = fmaxf(qmax, q[s]);
    }
    const float S = warp_sum(part);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qmax = fmaxf(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
    // uniform when every Q is below the smallest normal binary32 value
    const bool uniform = !(qmax >= 0x1p-126f) || !isfinite(S);
    const float add = eps * S / (float)m;
    const int ipl = (m + 31) >> 5;
    const int b = lane * ipl, e = min(m, b + ipl);
    float run = 0.0f;
    for (int s = b; s < e; ++s) {
        run += uniform ? 1.0f : q[s] + add;
        c[s] = run;
    }
    float x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const float before = x - run;
    for (int s = b; s < e; ++s) c[s] += before;
    __syncwarp();
    if constexpr (P == RLL_PREC_FP32) {
        for (int s = lane; s < m; s += 32) out[s] = Store<P>::store(c[s]);
        __syncwarp();
        return;
    } else {
        const float total = c[m - 1];
        for (int s = lane; s < m; s += 32) bits[s] = Store<P>::bits(Store<P>::store(c[s] / total));
        __syncwarp();
        // Strictly increasing bit patterns (positive values order as their bits), last = 1.0:
        // forward, b[s] = max(b[s], b[s-1] + 1) for s < m - 1 (b[-1] = 0); then b[m-1] = one;
        // backward, b[s] = min(b[s], b[s+1] - 1) for s = m - 2 .. 0. Both recurrences are
        // scans: b'[s] - s is the running maximum of b[t] - t (at least 1), and b''[s] - s the
        // running minimum of b'[t] - t from the top, so each lane scans its `ipl` entries and
        // the lanes combine by shuffles. The patterns stay within 1 .. one (m <= 256), so the
        // 16-bit values never wrap and the result equals the sequential loops.
        const int one = Store<P>::bits(Store<P>::store(1.0f));
        constexpr int kIpl = kMaxCut / 32;  // entries a lane holds at most
        int mx = INT_MIN;
#pragma unroll
        for (int j = 0; j < kIpl; ++j) {
            const int s = b + j;
            if (s < e && s < m - 1) mx = max(mx, (int)bits[s] - s);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, mx, o);
            if (lane >= o) mx = max(mx, y);
        }
        int up = __shfl_up_sync(0xffffffffu, mx, 1);
        up = lane == 0 ? 1 : max(up, 1);
#pragma unroll
        for (int j = 0; j < kIpl; ++j) {
            const int s = b + j;
            if (s < e && s < m - 1) {
                up = max(up, (int)bits[s] - s);
                bits[s] = (uint16_t)(s + up);
            }
        }
        if (b <= m - 1 && m - 1 < e) bits[m - 1] = (uint16_t)one;
        int mn = INT_MAX;
#pragma unroll
        for (int j = kIpl - 1; j >= 0; --j) {
            const int s = b + j;
            if (s < e) mn = min(mn, (int)bits[s] - s);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_down_sync(0xffffffffu, mn, o);
            if (lane + o < 32) mn = min(mn, y);
        }
        int down = __shfl_down_sync(0xffffffffu, mn, 1);
        if (lane == 31) down = INT_MAX;
#pragma unroll
        for (int j = kIpl - 1; j >= 0; --j) {
            const int s = b + j;
            if (s < e) {
                down = min(down, (int)bits[s] - s);
                bits[s] = (uint16_t)(s + down);
            }
        }
        __syncwarp();
        for (int s = lane; s < m; s += 32) out[s] = Store<P>::from_bits(bits[s]);
        __syncwarp();
    }
}

struct ArgBest {
    float v;
    uint32_t i;
};

__device__ __forceinline__ ArgBest warp_argmax(ArgBest a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, a.v, o);
        const uint32_t i = __shfl_xor_sync(0xffffffffu, a.i, o);
        if (i != 0xFFFFFFFFu && (a.i == 0xFFFFFFFFu || v > a.v || (v == a.v && i < a.i))) {
            a.v = v;
            a.i = i;
        }
    }
    return a;
}

__device__ __forceinline__ ArgBest warp_argmin(ArgBest a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, a.v, o);
        const uint32_t i = __shfl_xor_sync(0xffffffffu, a.i, o);
        if (i != 0xFFFFFFFFu && (a.i == 0xFFFFFFFFu || v < a.v || (v == a.v && i < a.i))) {
            a.v = v;
            a.i = i;
        }
    }
    return a;
}

// Eq. 1 for one cell: walk the cell's sorted records from `start` 32 at a
// time; a segmented inclusive scan (by cluster) composes the affine maps
// q -> (1 - alpha) q + alpha |c| in sample order and the last lane of each
// segment applies the composite to the cluster's Q. Then the row is stored
// in the table precision and its cdf rebuilt (Eq. 2). `key` tells whether a
// record belongs to the cell (same()) and its cluster (cluster()).
template <int P, class Key>
__device__ void learn_one_cell(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv, int64_t n,
                               int64_t start, const Key& key, typename Store<P>::T* qrow,
                               typename Store<P>::T* crow, uint32_t m, float alpha, float eps, float* q, float* c,
                               uint16_t* bits)
{
    const int lane = threadIdx.x & 31;
    const float a1 = 1.0f - alpha;
    for (uint32_t s = lane; s < m; s += 32) q[s] = Store<P>::load(qrow[s]);
    __syncwarp();
    for (int64_t pos = start;; pos += 32) {
        const int64_t i = pos + lane;
        const uint32_t k = i < n ? sk[i] : 0xFFFFFFFFu;
        const bool valid = i < n && key.same(k);
        const uint32_t mask = __ballot_sync(0xffffffffu, valid);
        if (!mask) break;
        const uint32_t s = valid ? key.cluster(k) : 0xFFFFFFFFu;
        float A = valid ? a1 : 1.0f;
        float B = valid ? alpha * __uint_as_float(sv[i]) : 0.0f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ao = __shfl_up_sync(0xffffffffu, A, o);
            const float Bo = __shfl_up_sync(0xffffffffu, B, o);
            const uint32_t so = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o && so == s) {
                B = A * Bo + B;
                A = A * Ao;
            }
        }
        const uint32_t s_next = __shfl_down_sync(0xffffffffu, s, 1);
        const bool last = valid && (lane == 31 || s_next != s);
        if (last && s < m) q[s] = A * q[s] + B;
        __syncwarp();
        if (mask != 0xffffffffu) break;
    }
    for (uint32_t s = lane; s < m; s += 32) {
        const typename Store<P>::T st = Store<P>::store(q[s]);
        qrow[s] = st;
        q[s] = Store<P>::load(st);
    }
    __syncwarp();
    warp_rebuild_cdf<P>(q, (int)m, eps, crow, c, bits);
}

// ---------------------------------------------------------------- per-cell sort
// Ascending sort of a[0..n) by a bitonic network in which every comparator
// puts the minimum at the lower index: per merge size k, first the mirror
// step (i against i ^ (k - 1)), then half-cleaners (i against i + j). The
// array is padded virtually to the next power of two with +infinity; a
// comparator that reaches a padded position would leave it unchanged, so it
// is skipped. `tid`/`nthreads` split the comparators; `sync` is the barrier
// of the participating threads (__syncwarp or __syncthreads).
__device__ __forceinline__ void cmp_swap(unsigned long long* a, uint32_t i, uint32_t p)
{
    const unsigned long long x = a[i], y = a[p];
    if (y < x) {
        a[i] = y;
        a[p] = x;
    }
}

template <class Sync>
__device__ __forceinline__ void bitonic_sort_u64(unsigned long long* a, uint32_t n, uint32_t tid, uint32_t nthreads,
                                                 Sync sync)
{
    if (n < 2) return;
    uint32_t lg = 0;
    while ((1u << lg) < n) ++lg;
    const uint32_t half_len = 1u << (lg - 1);
    for (uint32_t lk = 1; lk <= lg; ++lk) {
        const uint32_t k = 1u << lk;
        for (uint32_t t = tid; t < half_len; t += nthreads) {
            const uint32_t i = ((t >> (lk - 1)) << lk) | (t & ((k >> 1) - 1));
            const uint32_t p = i ^ (k - 1);
            if (p < n) cmp_swap(a, i, p);
        }
        sync();
        for (uint32_t lj = lk - 1; lj-- > 0;) {
            const uint32_t j = 1u << lj;
            for (uint32_t t = tid; t < half_len; t += nthreads) {
                const uint32_t i = ((t >> lj) << (lj + 1)) | (t & (j - 1));
                const uint32_t p = i + j;
                if (p < n) cmp_swap(a, i, p);
            }
            sync();
        }
    }
}

// Eq. 1 for one cell whose records are given in (cluster, sample id) order:
// get(j) = (cluster, reward bits) of record j < len. The records are
// composed 32 at a time exactly as learn_one_cell does (segmented scan of the
// affine maps, in sample order per cluster), so both give the same bits.
// q: the warp's shared Q row. Does not store the row. All 32 lanes call it.
template <int P, class Get>
__device__ void learn_records(Get get, uint32_t len, uint32_t m, float alpha, float* q)
{
    const int lane = threadIdx.x & 31;
    const float a1 = 1.0f - alpha;
    for (uint32_t pos = 0; pos < len; pos += 32) {
        const uint32_t j = pos + lane;
        const bool valid = j < len;
        const uint2 e = valid ? get(j) : make_uint2(0xFFFFFFFFu, 0u);
        const uint32_t s = e.x;
        float A = valid ? a1 : 1.0f;
        float B = valid ? alpha * __uint_as_float(e.y) : 0.0f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ao = __shfl_up_sync(0xffffffffu, A, o);
            const float Bo = __shfl_up_sync(0xffffffffu, B, o);
            const uint32_t so = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o && so == s) {
                B = A * Bo + B;
                A = A * Ao;
            }
        }
        const uint32_t s_next = __shfl_down_sync(0xffffffffu, s, 1);
        const bool last = valid && (lane == 31 || s_next != s);
        if (last && s < m) q[s] = A * q[s] + B;
        __syncwarp();
    }
}

// Split-collapse steps on one cell's rows in shared memory (cut cs, Q q,
// both of m entries; c and nc: scratch rows), repeated until a step changes
// nothing or max_iter steps were taken; returns the number of steps taken.
// New Q values in correctly rounded binary32, then rounded to the table
// precision: l_max's Q times f = phi_a / (phi_a + phi_c) and times 1 - f
// (children's power), p_min's Q the sum of its children's. One warp.
template <int P>
__device__ uint32_t split_collapse_steps(uint32_t* cs, float* q, float* c, uint32_t* nc, uint32_t m,
                                const NodeRec* __restrict__ nodes, const int32_t* __restrict__ parent,
                                const int32_t* __restrict__ left, const int32_t* __restrict__ right, float T,
                                uint32_t max_iter, int64_t n_nodes)
{
    const int lane = threadIdx.x & 31;
    const uint32_t n_internal = (uint32_t)((n_nodes - 1) / 2);  // ids below are internal nodes
    uint32_t steps = 0;
    for (; steps < max_iter; ++steps) {
        ArgBest hi{0.0f, 0xFFFFFFFFu}, lo{0.0f, 0xFFFFFFFFu};
        for (uint32_t s = lane; s < m; s += 32) {
            if (cs[s] < n_internal && (hi.i == 0xFFFFFFFFu || q[s] > hi.v)) {
                hi.v = q[s];
                hi.i = s;
            }
            if (s + 1 < m) {
                const int32_t pa = parent[cs[s]];
                if (pa >= 0 && pa == parent[cs[s + 1]]) {
                    const float v = fadd(q[s], q[s + 1]);
                    if (lo.i == 0xFFFFFFFFu || v < lo.v) {
                        lo.v = v;
                        lo.i = s;
                    }
                }
            }
        }
        hi = warp_argmax(hi);
        lo = warp_argmin(lo);
        const bool apply = hi.i != 0xFFFFFFFFu && lo.i != 0xFFFFFFFFu && hi.i != lo.i && hi.i != lo.i + 1 &&
                           hi.v > fmul(T, lo.v);
        if (!apply) break;
        // the new row into the scratch rows nc / c, every lane placing its own entries: entry i
        // moves to i + [i > hi] - [i > lo + 1] (one more before it after the split, one fewer
        // after the merge); hi becomes its two children, lo and lo + 1 their parent
        const uint32_t H = hi.i, L = lo.i;
        const uint32_t node = cs[H];
        const uint32_t a = (uint32_t)left[node], cc = (uint32_t)right[node];
        const float pa = nodes[a].phi, pc = nodes[cc].phi;
        const float sum = fadd(pa, pc);
        const float fa = sum > 0.0f ? fdiv(pa, sum) : 0.5f;
        float* nq = c;
        for (uint32_t i = lane; i < m; i += 32) {
            if (i == L + 1) continue;
            const uint32_t k = i + (i > H ? 1u : 0u) - (i > L + 1 ? 1u : 0u);
            if (i == H) {
                nc[k] = a;
                nq[k] = Store<P>::load(Store<P>::store(fmul(q[i], fa)));
                nc[k + 1] = cc;
                nq[k + 1] = Store<P>::load(Store<P>::store(fmul(q[i], fsub(1.0f, fa))));
            } else if (i == L) {
                nc[k] = (uint32_t)parent[cs[i]];
                nq[k] = Store<P>::load(Store<P>::store(fadd(q[i], q[i + 1])));
            } else {
                nc[k] = cs[i];
                nq[k] = q[i];
            }
        }
        __syncwarp();
        for (uint32_t i = lane; i < m; i += 32) {
            cs[i] = nc[i];
            q[i] = nq[i];
        }
        __syncwarp();
    }
    return steps;
}

// Loads cut row crow into cs (m entries); false (and RLL_E_DEVICE flagged)
// when an entry is not a node of the tree. One warp.
__device__ __forceinline__ bool load_cut_row(const uint32_t* crow, uint32_t* cs, uint32_t m, int64_t n_nodes,
                                             uint32_t* status)
{
    const int lane = threadIdx.x & 31;
    bool bad = false;
    for (uint32_t s = lane; s < m; s += 32) {
        cs[s] = crow[s];
        bad |= (int64_t)cs[s] >= n_nodes;
    }
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) atomicOr(status, (uint32_t)RLL_E_DEVICE);
        return false;
    }
    __syncwarp();
    return true;
}

// Split-collapse of one cell (cut row crow, Q row qrow, cdf row ccrow): the
// steps above on the rows loaded into shared memory; when a step was taken,
// the rows are stored and C rebuilt (Eq. 2). A corrupt cut row is flagged
// and the cell left alone. One warp; q, c, cs, nc, bits: its scratch rows.
template <int P>
__device__ void split_one_cell(uint32_t* crow, typename Store<P>::T* qrow, typename Store<P>::T* ccrow, uint32_t m,
                               const NodeRec* __restrict__ nodes, const int32_t* __restrict__ parent,
                               const int32_t* __restrict__ left, const int32_t* __restrict__ right, float T,
                               float eps, uint32_t max_iter, int64_t n_nodes, uint32_t* status, float* q, float* c,
                               uint32_t* cs, uint32_t* nc, uint16_t* bits)
{
    const int lane = threadIdx.x & 31;
    if (!load_cut_row(crow, cs, m, n_nodes, status)) return;
    for (uint32_t s = lane; s < m; s += 32) q[s] = Store<P>::load(qrow[s]);
    __syncwarp();
    const uint32_t steps = split_collapse_steps<P>(cs, q, c, nc, m, nodes, parent, left, right, T, max_iter, n_nodes);
    if (steps == 0) return;
    for (uint32_t s = lane; s < m; s += 32) {
        crow[s] = cs[s];
        qrow[s] = Store<P>::store(q[s]);  // exact: q holds table values
    }
    __syncwarp();
    warp_rebuild_cdf<P>(q, (int)m, eps, ccrow, c, bits);
}

}  // namespace rll
