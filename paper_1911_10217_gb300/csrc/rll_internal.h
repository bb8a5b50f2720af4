// Host-side state behind the opaque handles of rll.h, and the launchers each
// translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rll.h"

namespace rll {
struct NodeRec;
struct DescRec;
struct PairRec;
struct LightRec;
}  // namespace rll

#define RLL_HOST_MAX_CHUNKS 32

struct rll_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t* d_status = nullptr;   // device status bits (RLL_E_* >= RLL_E_TABLE_FULL)
    std::string err;
    // growable library-owned scratch (sort buffers, staging)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // staging for rll_render_pass_host
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // rll_render_pass_host pipeline: upload, download and second compute
    // streams, and its events (created on first use)
    cudaStream_t up = nullptr, down = nullptr, comp2 = nullptr;
    cudaEvent_t ev[2 * RLL_HOST_MAX_CHUNKS + 3] = {};
    bool pipe_ready = false;
    int host_chunks = 8;
    int host_zero_copy = 1;  // rll_render_pass_host: use mapped host buffers in place
    // launch tuning (rll_ctx_set_option)
    int sample_min_blocks = 4;
    // occluder boxes sorted by their lower x bound, then their widest x extent, rebuilt by every
    // sampling call (sample.cu: sort_boxes); allocated on first use
    void* box_sorted = nullptr;
};

struct rll_tree {
    int device = 0;
    int64_t n = 0;
    rll::NodeRec* nodes = nullptr;   // [2n-1] every node
    rll::PairRec* pairs = nullptr;   // [n-1] descent records of both children of internal i, interleaved
    rll::DescRec* quads = nullptr;   // [4(n-1)] records of the 2..4 grandchildren of internal i at 4i.. (two-level
                                     // descent; a single-light child stands for itself; unused entries id ~0)
    rll::LightRec* lights = nullptr; // [n] sorted lights
    uint32_t* perm = nullptr;        // [n] sorted -> input index
    int32_t* left = nullptr;         // [n-1]
    int32_t* right = nullptr;        // [n-1]
    int32_t* parent = nullptr;       // [2n-1]
    float* light_cdf = nullptr;      // [n] inclusive prefix of leaf power (energy sampler)
};

struct rll_grid {
    int device = 0;
    rll_grid_params p{};
    uint32_t H = 0, M = 0, m = 0;   // H: slots of all levels (levels * Hl)
    uint32_t Hl = 0, levels = 1;    // slots per resolution level, levels
    int64_t n_lights = 0;
    unsigned long long* keys = nullptr;  // [H]
    uint32_t* cut = nullptr;             // [H*M]
    void* Q = nullptr;                   // [H*M] table precision
    void* C = nullptr;                   // [H*M] table precision
    uint32_t* def_cut = nullptr;         // [m]
    void* def_Q = nullptr;               // [m]
    void* def_C = nullptr;               // [m]
    uint32_t* touched = nullptr;         // [H] cells touched by the last learn_update
    uint32_t* touched_start = nullptr;   // [H] first record of each touched cell (sorted / bucketed)
    uint32_t* touched_len = nullptr;     // [H] records of each touched cell (bucketed learning)
    uint32_t* n_touched = nullptr;       // [8]: touched cells, bucket space claimed, sorting- and grouping-path
                                         // cells, two work counters of the learning kernel
    uint32_t* cursor = nullptr;          // [H] per-slot record count / scatter cursor, all zero between calls
    uint32_t* big = nullptr;             // [2H] touched-cell indices for the grouping, then the sorting block path
    bool cursor_dirty = false;           // a learning call stopped before the cursors were cleared
};

namespace rll {

// Makes `dev` the current device for the guard's lifetime (restores the
// previous one).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// status helpers (api.cu)
int fail(rll_ctx* ctx, int code, const std::string& msg);
int check_cuda(rll_ctx* ctx, cudaError_t e, const char* what);
void* ws_get(rll_ctx* ctx, size_t bytes);  // nullptr on failure (error recorded)

// ---- sort.cu
// Scratch of radix_sort_pairs for n items: four key/value arrays, the
// per-tile digit counts (up to 512 digits, tiles of 2048) and the digit
// totals, each rounded up to 256 bytes.
constexpr int kSortTile = 2048;
constexpr int kSortMaxDigits = 512;
constexpr size_t sort_align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t sort_scratch_bytes_for(int64_t n)
{
    return 4 * sort_align256(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)) +
           sort_align256(sizeof(uint32_t) * kSortMaxDigits * (size_t)(n > 0 ? (n + kSortTile - 1) / kSortTile : 1)) +
           sort_align256(sizeof(uint32_t) * kSortMaxDigits);
}
size_t radix_sort_scratch_bytes(int64_t n);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of
// min(key, clamp). Input arrays are not modified; the sorted arrays are
// written to scratch and returned through kout / vout.
cudaError_t radix_sort_pairs(cudaStream_t s, const uint32_t* kin, const uint32_t* vin, int64_t n,
                             int bits, uint32_t clamp, void* scratch, uint32_t** kout,
                             uint32_t** vout);
// Inclusive prefix sum of n floats (n <= 2^24) into out; scratch >= 4 * 4096 bytes.
cudaError_t inclusive_scan_f32(cudaStream_t s, const float* in, float* out, int64_t n, void* scratch);

// ---- tree.cu
int build_tree(rll_ctx* ctx, const float* tri, const float* emission, int64_t n, int builder, rll_tree* t);
int tree_update_emission(rll_ctx* ctx, rll_tree* t, const float* emission);

// ---- learn.cu
int grid_init(rll_ctx* ctx, rll_grid* g);
int grid_to_float(rll_ctx* ctx, const rll_grid* g, float* q_out, float* c_out);   // device out
int grid_from_float(rll_ctx* ctx, rll_grid* g, const float* q_in, const float* c_in); // device in
int grid_mark_occupied(rll_ctx* ctx, rll_grid* g);  // touched list := every occupied slot
int key_bits(uint64_t hm_plus_one);
int device_sm_count(int device);
// split-collapse steps per cell and call (0 reads as 1)
inline uint32_t split_steps(const rll_grid_params& p) { return p.split_iterations ? p.split_iterations : 1u; }
int learn_update(rll_ctx* ctx, rll_grid* g, const uint32_t* rec_key, const float* rec_val, int64_t n);
int split_collapse(rll_ctx* ctx, rll_grid* g, const rll_tree* t);
// learn_update followed by split_collapse, fused per cell (same tables)
int learn_update_split(rll_ctx* ctx, rll_grid* g, const rll_tree* t, const uint32_t* rec_key, const float* rec_val,
                       int64_t n);
// learn_update with the sort buffers in caller-provided device scratch
int learn_update_with_scratch(rll_ctx* ctx, rll_grid* g, const uint32_t* rec_key, const float* rec_val, int64_t n,
                              void* scratch, size_t scratch_bytes);

// ---- sample.cu
int sample_and_shade(rll_ctx* ctx, rll_grid* g, const rll_tree* t, const float* pos, const float* nrm,
                     const float* albedo, const float* footprint, int64_t n_points, const float* boxes, int n_boxes,
                     uint64_t seed, uint32_t frame, int spp, float* rgb, uint32_t* rec_key,
                     float* rec_val, const rll_sample_debug* dbg);
// Shades points [p_begin, p_end) of a G-buffer of n_points (the plane stride)
// on `stream`; sample ids, records and rgb are those of the whole launch.
// The boxes sorted for sample_and_shade_range (enqueued on `stream`); returns the device
// buffer through *out (nullptr when there are no boxes).
int sort_boxes(rll_ctx* ctx, const float* boxes, int n_boxes, cudaStream_t stream, const void** out);
int sample_and_shade_range(rll_ctx* ctx, rll_grid* g, const rll_tree* t, const float* pos, const float* nrm,
                           const float* albedo, const float* footprint, int64_t n_points, int64_t p_begin,
                           int64_t p_end, const float* boxes, int n_boxes, uint64_t seed, uint32_t frame, int spp,
                           float* rgb, uint32_t* rec_key, float* rec_val, const rll_sample_debug* dbg,
                           cudaStream_t stream, const void* sorted_boxes);
int sample_power(rll_ctx* ctx, const rll_tree* t, const float* pos, const float* nrm,
                 const float* albedo, int64_t n_points, const float* boxes, int n_boxes, uint64_t seed,
                 uint32_t frame, int spp, float* rgb, int32_t* light_out);

}  // namespace rll
