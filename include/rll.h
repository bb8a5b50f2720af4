/*
 * rll.h -- C ABI of the GB300 (sm_103a) implementation of Reinforcement
 * Lightcuts Learning (Pantaleoni, arXiv 1911.10217).
 *
 * Conventions for every entry point:
 *  - Bulk arrays are plain pointers to DEVICE memory owned by the caller
 *    (e.g. contiguous torch tensors), unless an argument says "host".
 *    Layouts are stated per argument; "SoA [3][P]" means all x, then all y,
 *    then all z.
 *  - rll_ctx, rll_tree and rll_grid are opaque handles owned by the library
 *    and released with the matching *_destroy call.
 *  - Work is enqueued on the context's CUDA stream and returns without
 *    waiting, except where a call says it synchronises.
 *  - The return value is a status code (RLL_OK = 0). A failing call leaves a
 *    message in rll_last_error(ctx). No C++ exception crosses this boundary.
 *    Problems found on the device (hash table full, a bounds check) set bits
 *    in a device status word that rll_sync_status() returns and clears.
 *  - Not thread-safe per context: one host thread drives one context.
 */
#ifndef RLL_H
#define RLL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RLL_OK 0
#define RLL_E_INVALID 1     /* bad argument (null pointer, size out of range) */
#define RLL_E_NOMEM 2       /* device allocation failed */
#define RLL_E_CUDA 3        /* a CUDA runtime call failed */
#define RLL_E_TABLE_FULL 4  /* device: a hash lookup hit the probe limit (sample used the initial cut) */
#define RLL_E_TIMEOUT 8     /* device: a bounded wait gave up */
#define RLL_E_DEVICE 16     /* device: an index failed its bounds check */

/* table precision of Q and C */
#define RLL_PREC_FP32 0
#define RLL_PREC_FP16 1
#define RLL_PREC_BF16 2

/* choice of a light inside the sampled cluster */
#define RLL_MODE_DESCENT 0  /* stochastic descent by unoccluded bounds (default) */
#define RLL_MODE_UNIFORM 1  /* uniform over the cluster's lights (Section 3 picks the light in the cluster at random) */
#define RLL_MODE_DESCENT2 2 /* descent two levels at a time: from a node, one of the children of its children (a
                               single-light child standing for itself) by their bounds (num / max(den, 1e-30));
                               the binary32 prefix sums P_i decide: first i with u * P_last < P_i, probability
                               (P_i - P_{i-1}) / P_last; powers, then uniform, when all bounds vanish */

/* the |c| fed to Eq. 1 */
#define RLL_REWARD_CLUSTER 0 /* luminance of c / (p_in * p_area): the cluster's contribution estimate (default) */
#define RLL_REWARD_LITERAL 1 /* luminance of c / p_area: the selected light's contribution */

typedef struct rll_ctx rll_ctx;
typedef struct rll_tree rll_tree;
typedef struct rll_grid rll_grid;

/* Parameters of a hash grid (Section 3: 5-d hash table, fixed-size cuts,
 * Q and C tables, Eq. 1 and Eq. 2, split-collapse threshold). */
typedef struct rll_grid_params {
    uint32_t table_size;       /* H slots, a power of two, 2^4 .. 2^26 */
    uint32_t cut_size;         /* M leaves per cut, 1 .. 256 (min(M, lights) are used) */
    float origin[3];           /* grid origin */
    float cell_size;           /* h: position quantisation step, > 0 */
    uint32_t normal_bins;      /* bins per octahedral normal axis, 1 .. 255 */
    uint32_t jitter;           /* 1: jitter every lookup by +-1/2 cell / bin (Section 3) */
    uint32_t precision;        /* RLL_PREC_* for stored Q and C */
    uint32_t in_cluster_mode;  /* RLL_MODE_* */
    uint32_t reward_mode;      /* RLL_REWARD_* */
    float alpha;               /* Eq. 1 learning rate, [0, 1] */
    float threshold;           /* split-collapse T (> 0) */
    float eps;                 /* Eq. 2 floor: eps * sum(Q) / m added to each leaf, >= 0 */
    float q_init;              /* Q of a new cell's leaves, > 0 */
    uint32_t split_iterations; /* split-collapse steps per cell and call, 1 .. 256 (0 reads as 1):
                                  1 is the basic algorithm; more repeat it until a step
                                  changes nothing (Section 3) */
    uint32_t levels;           /* resolution levels, 1 .. 16 (0 reads as 1). Section 3 sizes the
                                  cells of a path vertex from its ray footprint (coarser for later
                                  bounces); here level l has cell size cell_size * 2^l and a table of
                                  its own of table_size slots (levels * table_size in all, at most
                                  2^27, and that times cut_size at most 2^31). A point with footprint
                                  f (rll_sample_and_shade_fp) uses the smallest level whose cell is
                                  at least f wide: l = ceil(log2(f / cell_size)) from the binary32
                                  quotient, clamped to [0, levels - 1]; f <= cell_size, NaN or no
                                  footprint give level 0. Slots of level l are l * table_size ..
                                  (l + 1) * table_size - 1 in record keys and exports. */
} rll_grid_params;

/* Per-sample diagnostics (optional outputs of rll_sample_and_shade_ex), each
 * [P * spp] in sample order (sample id = point * spp + j); any may be NULL. */
typedef struct rll_sample_debug {
    int32_t* light;            /* sorted light index chosen */
    float* p_cut;              /* probability of the chosen cluster */
    float* p_in;               /* probability of the light inside the cluster */
} rll_sample_debug;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on `device` that enqueues on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). */
int rll_ctx_create(rll_ctx** out, int device, void* cuda_stream);
int rll_ctx_set_stream(rll_ctx* ctx, void* cuda_stream);
/* Launch tuning of this context (no effect on results):
 *   "sample_min_blocks" 3 | 4 -- register budget of the sampling kernel:
 *   4 = 64 registers (8 resident 128-thread blocks, 32 warps per SM; the
 *   default), 3 = 80 registers (6 blocks, 24 warps);
 *   "host_chunks" 1..32 -- chunks rll_render_pass_host cuts the points into
 *   for copy/compute overlap (default 8; sizes growing by 3/2, at least 4 096
 *   points each);
 *   "host_zero_copy" 0 | 1 -- rll_render_pass_host uses mapped host buffers
 *   in place (default 1).
 * Returns RLL_E_INVALID for an unknown name or a value out of range. */
int rll_ctx_set_option(rll_ctx* ctx, const char* name, int64_t value);
int rll_ctx_destroy(rll_ctx* ctx);
/* Message of the last failing call on this context ("" if none). */
const char* rll_last_error(const rll_ctx* ctx);
/* Synchronises the stream, returns the OR of device status bits raised since
 * the last call (0 = none) and clears them. Returns a negative value if the
 * synchronisation itself failed. */
int rll_sync_status(rll_ctx* ctx);

/* ---- light tree (Section 3, Section 3.1: sort the lights, one binary tree
 * over all of them, built as an LBVH over light positions) ---------------- */

/* Builds the tree over n triangles. tri: [n][3][3] float (v0, v1, v2);
 * emission: [n][3] RGB radiance used for the node power bounds (pass the
 * maximum over time for changing lights). Lights are sorted by the 30-bit
 * Morton code of their centroid, ties by input index; node numbering:
 * internal nodes 0..n-2, the leaf of sorted light l is n-1+l, root 0.
 * Triangles must have non-zero area. n in [1, 2^24]. Synchronises. */
int rll_build_light_tree(rll_ctx* ctx, const float* tri, const float* emission, int64_t n,
                         rll_tree** out);

/* tree builders (rll_build_light_tree_ex) */
#define RLL_TREE_LBVH 0  /* radix tree of the Morton codes (Section 3.1: a simple LBVH) */
#define RLL_TREE_SAOH 1  /* same light order, split positions by a surface-area-orientation cost */
#define RLL_TREE_MEDIAN 2 /* same light order, every range split at its middle (balanced) */

/* Same, with a choice of builder. RLL_TREE_SAOH follows the alternative that
 * Section 3.1 leaves as future work (a hierarchy that considers light
 * orientations and a surface area heuristic): the lights keep their Morton
 * order, so every node is still a contiguous range; each node's split
 * position is, among every position (ranges of at most 17 lights) or the 15
 * positions b + floor(m j / 16) and the Morton split, the one of least
 * cost(L) + cost(R), ties to the smallest, where cost(S) = phi(S) *
 * surface area of S's box * (2 - |sum of winding cross products| / sum of
 * their lengths); power, lengths and cross products are summed in 64-bit
 * fixed point, so the result does not depend on summation order. Internal
 * node ids are (split position - the root's) mod (n - 1): root 0.
 * RLL_TREE_MEDIAN: same light order and id rule, every range [b, e) of at
 * least two lights split at b + floor((e - b) / 2), so every leaf lies at
 * depth floor(log2 n) or ceil(log2 n). Same output layout and export as
 * rll_build_light_tree. RLL_E_INVALID for another builder. Synchronises. */
int rll_build_light_tree_ex(rll_ctx* ctx, const float* tri, const float* emission, int64_t n,
                            int32_t builder, rll_tree** out);
/* Replaces the radiance used for shading (emission: [n][3], input order);
 * the node power bounds keep the values given at build time. */
int rll_tree_update_emission(rll_ctx* ctx, rll_tree* tree, const float* emission);
int64_t rll_tree_num_lights(const rll_tree* tree);
/* Copies the tree to HOST arrays (any may be NULL): perm [n] sorted->input
 * index, left/right [n-1], parent [2n-1] (-1 at root), begin/end [2n-1],
 * rec [2n-1][11] = bmin xyz, bmax xyz, power, cone axis xyz, cone cos.
 * Synchronises. */
int rll_tree_export(rll_ctx* ctx, const rll_tree* tree, uint32_t* perm, int32_t* left,
                    int32_t* right, int32_t* parent, uint32_t* begin, uint32_t* end, float* rec);
int rll_tree_destroy(rll_tree* tree);

/* ---- hash grid of learned cuts (Section 3) ------------------------------- */

/* Creates a grid whose every slot starts empty and holds the initial cut:
 * the breadth-first cut of min(M, n) nodes (Section 3), Q = q_init, C from
 * Eq. 2. Synchronises. */
int rll_create_grid(rll_ctx* ctx, const rll_tree* tree, const rll_grid_params* params,
                    rll_grid** out);
/* Number of leaves m = min(M, lights) in every cut. */
uint32_t rll_grid_cut_len(const rll_grid* grid);
/* Cells touched by the last learning call (rll_learn_update,
 * rll_learn_update_split, rll_learn_update_noalloc; after rll_grid_import:
 * every occupied cell), written to the HOST int64 *out. These are the cells
 * whose Q and C rows Eq. 1 and Eq. 2 rewrote, the unit of the learning step's
 * table traffic. Synchronises. */
int rll_grid_touched_cells(rll_ctx* ctx, const rll_grid* grid, int64_t* out);
/* Copies the grid to HOST arrays (any may be NULL): keys [H] (empty slots
 * 0xFFFFFFFFFFFFFFFF), cut [H][M] node ids, q and c [H][M] as float (16-bit
 * tables widened exactly). Only the first m entries of a row are meaningful.
 * Also the checkpoint format. Synchronises. */
int rll_grid_export(rll_ctx* ctx, const rll_grid* grid, uint64_t* keys, int32_t* cut, float* q,
                    float* c);
/* Loads a state written by rll_grid_export (HOST arrays, same shapes; q and c
 * are rounded to the table precision). Rows of empty slots are ignored and
 * reset to the initial cut. Every occupied slot becomes a touched cell, so a
 * following rll_split_collapse adapts all of them. Synchronises. */
int rll_grid_import(rll_ctx* ctx, rll_grid* grid, const uint64_t* keys, const int32_t* cut,
                    const float* q, const float* c);
int rll_grid_destroy(rll_grid* grid);

/* ---- one rendering pass: sampling (Section 3 / Section 3.1) ------------- */

/* For every shading point and sample: hash the (jittered) point to its cell
 * (creating it on first access), pick a cluster by binary search in C, a
 * light inside it (descent or uniform), a point on that triangle, and
 * evaluate the shadowed contribution against the boxes. Writes the
 * per-point mean estimate and one learning record per sample.
 * Visibility: the segment from x + 1e-4 n to the light point y, parameter
 * t in (0, 0.9999), misses every box (binary32 slab test, open intervals);
 * a segment that does not move along an axis (|y - o| < 2^-100 there) is
 * inside that axis's slab exactly when the box's open interval contains it.
 *   pos, nrm: SoA [3][P] float; albedo [P]; boxes [K][6] (min xyz, max xyz),
 *   K <= 1024; rgb: SoA [3][P] output; rec_key [P*spp]: slot * M + cluster
 *   (0xFFFFFFFF when no cell could be created); rec_val [P*spp]: |c| (Eq. 1
 *   reward). rec_key / rec_val may both be NULL (no learning).
 * Random numbers: Philox4x32-10, key = seed, counter = (point * spp + j,
 * frame, draw block, 0). P * spp < 2^32. Q and C are only read. */
int rll_sample_and_shade(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos,
                         const float* nrm, const float* albedo, int64_t n_points,
                         const float* boxes, int32_t n_boxes, uint64_t seed, uint32_t frame,
                         int32_t spp, float* rgb, uint32_t* rec_key, float* rec_val);
/* Same, with optional per-sample diagnostics (dbg may be NULL). */
int rll_sample_and_shade_ex(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos,
                            const float* nrm, const float* albedo, int64_t n_points,
                            const float* boxes, int32_t n_boxes, uint64_t seed, uint32_t frame,
                            int32_t spp, float* rgb, uint32_t* rec_key, float* rec_val,
                            const rll_sample_debug* dbg);

/* Same, with a footprint per point (footprint: [P] float, world units; NULL
 * = level 0 for every point): the point's samples use the grid level its
 * footprint selects (rll_grid_params.levels). Everything else as
 * rll_sample_and_shade_ex. */
int rll_sample_and_shade_fp(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos,
                            const float* nrm, const float* albedo, const float* footprint,
                            int64_t n_points, const float* boxes, int32_t n_boxes, uint64_t seed,
                            uint32_t frame, int32_t spp, float* rgb, uint32_t* rec_key,
                            float* rec_val, const rll_sample_debug* dbg);

/* Path vertices of one diffuse bounce and their footprints (Section 3, first
 * ingredient: a path vertex's cells are sized from its ray footprint, derived
 * from its area pdf). From every point x (pos, nrm: SoA [3][P], unit normals)
 * one cosine-weighted direction: a uniform point (a, b) of the unit disk by
 * rejection (Philox key = seed, counter = (point, frame, k / 2, 1), pair k =
 * words 2k mod 4 and 2k + 1 mod 4 as 2u - 1, the first of 16 pairs with
 * a^2 + b^2 < 1, else the centre), lifted to d = a u + b v + sqrt(1 - a^2 -
 * b^2) n with u = normalise(n x t), v = n x u, t the x axis (the z axis when
 * |n.x| >= 0.9). The ray from o = x + 1e-4 n meets the nearest surface ahead
 * (t > 1e-6): a box face (boxes [K][6], K <= 1024) or, from the inside, a wall
 * of the room (HOST float[6]: min xyz, max xyz). Outputs (device, caller
 * owned): out_pos SoA [3][P] the vertex y = o + t d, out_nrm SoA [3][P] the
 * hit face's axis normal turned toward x, out_footprint [P] =
 * t sqrt(pi / (N_t cos_x cos_y)) = (N_t p_A)^(-1/2), where p_A = cos_x cos_y
 * / (pi t^2) is the vertex's area density for one path, N_t = paths_per_tile
 * (> 0) the paths that leave one tile and share it, and each cosine is at
 * least 1e-6. A ray with nothing ahead (a point outside the room) escapes:
 * y = o, normal 0, footprint +inf (rll_sample_and_shade_fp then uses the
 * coarsest level). Every step is one correctly rounded binary32 operation.
 * P < 2^32. Enqueued on the context stream. */
int rll_bounce_vertices(rll_ctx* ctx, const float* pos, const float* nrm, int64_t n_points,
                        const float* boxes, int32_t n_boxes, const float* room, uint64_t seed,
                        uint32_t frame, float paths_per_tile, float* out_pos, float* out_nrm,
                        float* out_footprint);

/* Energy-based baseline (Section 4): lights chosen in proportion to their
 * emitted power by inversion of one global cdf; same shading, same Philox
 * stream (cluster draw reused as the cdf draw). rgb: SoA [3][P]. */
int rll_sample_power(rll_ctx* ctx, const rll_tree* tree, const float* pos, const float* nrm,
                     const float* albedo, int64_t n_points, const float* boxes, int32_t n_boxes,
                     uint64_t seed, uint32_t frame, int32_t spp, float* rgb, int32_t* light_out);

/* ---- end of pass: learning (Section 3, Eq. 1 and Eq. 2) ------------------ */

/* Applies Eq. 1, Q(s) := (1 - alpha) Q(s) + alpha |c|, for every record, in
 * sample order per (cell, cluster) -- a deterministic segmented reduction
 * (records bucketed by cell, each bucket ordered by (cluster, sample id),
 * then the affine updates composed per cluster) -- then rebuilds C of every
 * touched cell by Eq. 2 with the eps floor. Records with key 0xFFFFFFFF (or
 * any key >= slots * cut_size) are skipped. Remembers the touched cells for
 * rll_split_collapse. Uses library-owned scratch memory (17 bytes per
 * record, grown with cudaMalloc when needed). At most 2^32 - 1 records. */
int rll_learn_update(rll_ctx* ctx, rll_grid* grid, const uint32_t* rec_key, const float* rec_val,
                     int64_t n_records);

/* Same as rll_learn_update, for callers that cannot allocate device memory
 * while they run (a host that owns all device memory through its own pool,
 * an allocation budget enforced outside CUDA, a loop that must not
 * synchronise -- rll_learn_update grows its workspace with cudaFree and
 * cudaMalloc). Nothing is allocated: the sort buffers are one fixed device
 * array inside the library (about 18 MB, held on every GPU that loads the
 * library until exit). At most 1048576 records per call; more returns
 * RLL_E_INVALID without launching. The first call on a device looks up the
 * array's address: make it before any stream capture. The address is kept
 * for the process's life and does not survive a cudaDeviceReset of that
 * device (do not call this entry point after one). All calls share the
 * array, so calls that overlap on the GPU race: serialise them. The paper has
 * no counterpart of this entry point. */
int rll_learn_update_noalloc(rll_ctx* ctx, rll_grid* grid, const uint32_t* rec_key,
                             const float* rec_val, int64_t n_records);

/* rll_learn_update followed by rll_split_collapse, fused: each touched
 * cell's Eq. 1 update, split-collapse steps (on the Q values as stored in the
 * table precision) and one Eq. 2 rebuild run back to back in the learning
 * kernels, so the rows are read once and C is built once. Tables, cut rows
 * and the touched set afterwards are identical to those of the two calls.
 * Same arguments and errors as those two calls. Enqueued on the context
 * stream. */
int rll_learn_update_split(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const uint32_t* rec_key,
                           const float* rec_val, int64_t n_records);
/* Split-collapse (Section 3, Fig. "TreeCuts"; Section 3.1: one thread group
 * per cell) on every cell touched by the last rll_learn_update: split the
 * non-single-light leaf of largest Q into its children and collapse the
 * parent of two cut leaves of smallest Q if Q(l_max) > T * Q(p_min); then
 * rebuild C (Eq. 2). */
int rll_split_collapse(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree);

/* ---- many uneven scenes in one persistent launch per stage --------------- */

/* One scene of a batch: its grid and tree and one pass's inputs/outputs
 * (device pointers, layouts as in rll_sample_and_shade). */
typedef struct rll_batch_item {
    rll_grid* grid;
    const rll_tree* tree;
    const float* pos;          /* SoA [3][P] */
    const float* nrm;          /* SoA [3][P] */
    const float* albedo;       /* [P] */
    int64_t n_points;          /* P */
    const float* boxes;        /* [K][6] */
    int32_t n_boxes;           /* K <= 1024 */
    uint64_t seed;             /* Philox key of this scene */
    uint32_t frame;            /* frame of the first pass (advanced by one per pass) */
    int32_t spp;
    float* rgb;                /* SoA [3][P] output */
} rll_batch_item;

typedef struct rll_batch rll_batch;

/* Reserves a batch able to hold up to max_items scenes with at most
 * max_records samples and max_cells table slots in total (< 2^26); all
 * device buffers are allocated here, once (among them 32 KB per item for the
 * item's boxes sorted for the shadow test). */
int rll_batch_reserve(rll_ctx* ctx, int32_t max_items, int64_t max_records, int64_t max_cells,
                      rll_batch** out);
/* Sets the scenes of the next passes (all grids with the same table
 * precision and in-cluster mode, cut sizes <= 64, each grid at most once,
 * within the reserved capacity). Enqueues the upload of the descriptors on
 * the context stream from page-locked staging owned by the batch and returns
 * without waiting for the stream (it waits only if the previous upload from
 * that staging has not run yet); allocates nothing; drops a recorded graph. */
int rll_batch_set_items(rll_ctx* ctx, rll_batch* b, const rll_batch_item* items, int32_t n_items);
/* rll_batch_reserve for exactly these items, then rll_batch_set_items.
 *
 * One pass = sampling of every item by one persistent kernel that takes
 * tiles of points from a global counter, one sort of all records, Eq. 1 +
 * Eq. 2 for every touched cell, optional split-collapse, then each item's
 * frame += 1. Per scene the result equals a pass run for that scene alone
 * through the batch (records are keyed by scene). Synchronises. */
int rll_batch_create(rll_ctx* ctx, const rll_batch_item* items, int32_t n_items, rll_batch** out);
/* Sets the sampling tile (points per work item, 32..2^20) and the occupancy
 * target (3 | 4 resident 256-thread blocks per SM). Drops a recorded graph. */
int rll_batch_set_config(rll_ctx* ctx, rll_batch* b, int32_t tile_points, int32_t min_blocks);
/* Autotuner: times the sampling stage for every tile size in
 * {128 .. 8192} x occupancy {3, 4} (best of two timed runs after a warm-up)
 * and keeps the fastest; reports the choice through the optional outputs.
 * Runs sampling passes (hash cells may be created; Q and C are untouched).
 * Synchronises. */
int rll_batch_tune(rll_ctx* ctx, rll_batch* b, int32_t* tile_points_out, int32_t* min_blocks_out);
/* Enqueues one pass on the context stream. */
int rll_batch_run(rll_ctx* ctx, rll_batch* b, int32_t do_split);
/* Records one pass as a CUDA graph (on a stream of the batch's own) after
 * synchronising the context stream; rll_batch_launch replays it on the
 * context stream, each replay one pass with the next frame. */
int rll_batch_capture(rll_ctx* ctx, rll_batch* b, int32_t do_split);
int rll_batch_launch(rll_ctx* ctx, rll_batch* b);
int rll_batch_destroy(rll_batch* b);

/* ---- one whole pass from host memory ------------------------------------- */

/* One whole pass from HOST buffers: G-buffer pos/nrm SoA [3][P], albedo [P],
 * boxes [K][6], rgb out SoA [3][P]. Runs rll_sample_and_shade, then
 * rll_learn_update_split (do_split) or rll_learn_update. When pos, nrm,
 * albedo and rgb are page-locked host memory mapped into the device address
 * space (cudaHostAlloc / cudaHostRegister under unified addressing) and
 * "host_zero_copy" is on, the sampling kernel reads and writes them in place
 * over the host link; otherwise they are copied in chunks ("host_chunks"):
 * a chunk is shaded as soon as its upload ends and read back as soon as it
 * is shaded, on streams of the context's own, while later chunks upload
 * (pageable memory is correct but serialises the copies). Either way the
 * results are those of one rll_sample_and_shade launch on device copies.
 * Work enqueued earlier on the context stream comes first. Staging buffers
 * are owned by the context. Synchronises. */
int rll_render_pass_host(rll_ctx* ctx, rll_grid* grid, const rll_tree* tree, const float* pos,
                         const float* nrm, const float* albedo, int64_t n_points,
                         const float* boxes, int32_t n_boxes, uint64_t seed, uint32_t frame,
                         int32_t spp, int32_t do_split, float* rgb);

#ifdef __cplusplus
}
#endif

#endif /* RLL_H */
