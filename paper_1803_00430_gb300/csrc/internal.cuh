// internal.cuh -- data structures and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace rp {

// ---------------------------------------------------------------------------
// Scene in device memory.
//   nodes: 4 float4 per internal BVH node i (the two children's boxes are stored in
//          the parent):  [0] = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//                        [1] = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//                        [2] = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//                        [3] = (int c0, int c1, -, -)
//          child >= 0 is an internal node, child < 0 is triangle ~child (leaf order).
//          Node 0 is the root.  A one-triangle scene has no nodes.
//   tris:  3 float4 per triangle in leaf (Morton) order, the input vertices exactly:
//          [0] = (v0, material as int bits), [1] = (v1, original index as int bits),
//          [2] = (v2, 0)
//   materials: alpha, scattering, w_diff = s/sbar, w_spec = (1-s)/(1-sbar) [mat][B],
//          thr[mat] = ceil(sbar * 2^24) (diffuse if the 24-bit uniform is below it).
// ---------------------------------------------------------------------------
// node visits of one traversal query are capped at ITER_CAP_MULT x nodes + 64 (a
// query of a well-formed tree visits every node at most once)
constexpr int ITER_CAP_MULT = 4;

struct SceneView {
    const float4 *__restrict__ nodes;
    const float4 *__restrict__ tris;
    const float *__restrict__ alpha;
    const float *__restrict__ scat;
    const float *__restrict__ wdiff;
    const float *__restrict__ wspec;
    const uint32_t *__restrict__ thr;
    int num_tris;
    int num_nodes;
    int B;
    int iter_cap;   // node visits per traversal query before RP_ERR_TIMEOUT
    float tmin;     // self-intersection guard used by FP32 queries
    double tmin_d;  // the same guard for FP64 re-decisions
    float lo[3];    // bounding box of the vertices (cells of the shadow-ray order)
    float ext[3];
    const int *anc = nullptr;  // [num_tris] the node SHADOW_HINT_UP levels above each leaf (0: the root), or null
    const int *up = nullptr;   // [num_nodes] the node SHADOW_HINT_UP levels above each internal node, or null
};

// A shadow-ray packet that found a blocker leaves its warp a hint: the node this many
// levels above the blocking leaf, where the warp's next packet towards the same source
// (the neighbouring tile) starts its walk.
constexpr int SHADOW_HINT_UP = 3;

// One scene of a trace step.  A single-scene step is a batch of one job; a
// batched step runs many jobs (scenes, each with its own sources, listener and
// ray budget) in the same persistent launches.
struct SceneJob {
    SceneView sc;
    unsigned long long first_ray;  // id of the job's first primary
    unsigned long long num_rays;   // primaries of the first wave
    unsigned long long hit_off;    // first slot of the job's region of the reflection buffer
    unsigned long long hit_cap;    // slots in that region (num_rays * M)
    unsigned int scene_id;         // Philox counter word 1
    int S;                         // sources of the job
    int src_off;                   // global index of the job's first source
    int lis;                       // index of the job's listener in the position table
};

// Per-job state of one step (device memory, zeroed per step).
struct JobState {
    unsigned long long n_hits;      // stored reflections
    unsigned long long primaries;   // K over all waves; the job's H is divided by it
    unsigned long long wave_begin;  // first ray id of the current wave
    unsigned long long wave_count;  // primaries of the current wave
    unsigned long long item_off;    // first shadow item of the job
    unsigned long long hit_prefix;  // stored reflections of the earlier jobs
    unsigned long long segments;    // closest-hit rays traced (single-job steps, for the refill)
};

// A run of consecutive primaries of one job; the batched paths kernel hands out
// chunks in longest-processing-time order.
struct RayChunk {
    int job;
    int count;
    unsigned long long start;
};

// Global counters of one step (device memory, zeroed per step).
struct TraceCounters {
    unsigned long long next_ray;     // virtual ray index handed out in the current wave
    unsigned long long n_records;    // contribution records in the current chunk
    unsigned long long next_item;    // shadow items fetched in the current chunk
    unsigned long long n_rerun;      // shadow items queued for an FP64 decision (current chunk)
    unsigned long long total_items; // shadow items of the step (sum over jobs of shadow_items(hits, S))
    unsigned long long total_hits;  // stored reflections of the step (sum over jobs)
    // planned refill: candidate rays still needed (0 = planned), primaries and waves;
    // where the wave walk stopped (segments used, next wave's size, walk started)
    unsigned long long plan_need, plan_rays, plan_waves;
    unsigned long long plan_used, plan_count, plan_started;
    unsigned long long n_er;  // early reflections stored (rp_trace_er)
    // store passes of the planned refill: ~(lowest ray id whose reflection or record
    // found no slot), 0 if none; reflections of rays past the waves, left out of the order
    unsigned long long store_fail, dropped_hits;
};

// Contribution records: key = (global source - first source of the group) * T + bin,
// ray id, e[B] (row of B floats).
struct Records {
    uint32_t *key;
    uint32_t *rid;
    float *e;
    unsigned long long cap;
};

// Stored reflections for next-event estimation (structure of arrays).
struct Hits {
    float4 *p;      // hit point, path length to it in .w (FP32 part)
    float4 *plo;    // residuals: hit point and path length = p + plo in FP64
    float4 *n;      // normal facing the arriving ray, leaf triangle in .w (int bits)
    float *ws;      // [j * B + b] path weight after absorption times s_b
    uint32_t *rid;  // primary ray id
    unsigned long long cap;
};

// Early reflections (orders 1 .. min_order - 1, at most 2) kept for the early-path
// cache of rp_trace_er: the reflection as in Hits, and the leaf triangle of the path's
// previous reflection (-1 for order 1).  cap = 0: not kept (every other step).
struct EarlyHits {
    Hits hits = {nullptr, nullptr, nullptr, nullptr, nullptr, 0ull};
    int *prev = nullptr;
    unsigned long long cap = 0ull;
};

// Store passes of the planned refill keep what the candidates' paths give: reflections,
// records and statistics.  A candidate whose place in the waves is not yet known when it
// is traced (speculative) keeps its statistics in a slot of its own; once the waves are
// known, the slots of the rays inside them are added to the step's statistics and the
// rest are dropped, with their reflections and records.  Slot q holds the candidate
// first_ray + spec_lo + q.
struct SpecRays {
    double *late = nullptr;   // [cap][B] energy of source-sphere hits past the histogram
    double *L = nullptr;      // [cap] path length over the reflections
    double *t1 = nullptr;     // [cap] distance to the first reflection
    float *w = nullptr;       // [cap][B] band weights when the path ended
    float *absb = nullptr;    // [cap][B] absorbed weights
    uint32_t *esc = nullptr;  // [cap] 1: the path escaped, 0: it reached M reflections
    uint32_t *sph = nullptr;  // [cap] source-sphere hits
    uint32_t *rerun = nullptr;         // [cap] FP64 re-decisions of the closest hit
    rp_trace_stats *saved = nullptr;   // the statistics before the step (restored on a fallback)
    unsigned long long cap = 0;        // slots; 0: no store passes (the counting passes re-trace)
};
// bytes of the SpecRays arrays for `cap` slots and B bands (the saved statistics first)
inline size_t spec_bytes(unsigned long long cap, int B)
{
    return sizeof(rp_trace_stats) + (size_t)cap * ((size_t)B * (8 + 4 + 4) + 8 + 8 + 3 * 4);
}

struct TraceConsts {
    int S;           // sources of the group (keys and accumulation span them)
    int B, K, T, M, min_order, sh_order;
    float rate, c, rs;
    int flags;
};

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct BvhBuildArgs {
    const float *verts;
    const int32_t *tris;
    const int32_t *tri_mat;
    const float *alpha;
    const float *scat;
    int nv, nt, nmat, B;
    float ray_eps;
};

struct BvhOut {
    float4 *nodes;
    float4 *tris;
    float *alpha, *scat, *wdiff, *wspec;
    uint32_t *thr;
    float tmin;
    double tmin_d;
    float lo[3], hi[3];
    int max_depth;
    int *pleaf = nullptr;  // if set: [nt] parent node of each leaf (Morton order), kept for refits
    int *pint = nullptr;   // if set: [nt - 1] parent node of each internal node (-1: the root)
    int *anc = nullptr;    // if set: [nt] the node SHADOW_HINT_UP levels above each leaf (shadow-ray hints)
    int *up = nullptr;     // if set: [nt - 1] the node SHADOW_HINT_UP levels above each internal node
};

// Builds the BVH; all temporaries are allocated and freed inside.  Returns a
// cudaError_t; device-detected input errors go to *status.
cudaError_t build_bvh(const BvhBuildArgs &a, BvhOut &out, int *d_status, cudaStream_t st);

// The step's stored reflections sorted by cell (job, Morton code of the position on
// a 2^bits grid per axis over the job's scene box), so that the shadow rays a warp
// traces start close together and aim at the same source.  The records themselves
// are copied in that order (TraceWork::shits), so a warp's loads are contiguous.
struct HitOrder {
    uint32_t *cell;  // [total hits] cell of the flattened reflection f
    uint32_t *perm;  // [total hits] slot in Hits of the i-th reflection in cell order
    uint32_t *cnt;   // [ncells + 1] counts, then cursors
    int bits;        // code bits per job (near-cubic cells over the job's scene box)
    int ncells;      // njobs x 2^bits
};

// counts per tile of the scans, and the tile sums a scan of n counts needs
constexpr int SCAN_TILE = 4096;
inline unsigned long long scan_parts(unsigned long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// shadow items of a job with h stored reflections and S sources: tiles of 32
// reflections x S sources, a short last tile padded to 32 per source.  The tiles go in
// groups of SHADOW_TILE_GROUP, source-major inside a group, so that a warp's block of
// SHADOW_TILE_GROUP x 32 items is neighbouring tiles towards one source.
constexpr int SHADOW_TILE_GROUP = 32;
constexpr int SRC_HINT_STRIDE = 8;  // ints between two sources' hints (one 32-byte sector each)
__host__ __device__ inline unsigned long long shadow_items(unsigned long long h, int S)
{
    return ((h + 31ull) / 32ull) * 32ull * (unsigned long long)S;
}

// Code bits per job of the reflection order (cells = njobs << bits): the cells of all
// jobs together stay within 2^cells_log2, with at least 3 bits per job.  22 gives a
// job alone 2^22 cells (about 0.15 m cubes over a 40 x 30 x 12 m hall).
inline int hit_order_bits(int njobs, int cells_log2 = 22)
{
    int lg = 0;
    while ((1ll << lg) < (long long)std::max(njobs, 1)) ++lg;
    return std::max(3, cells_log2 - lg);
}
inline long long hit_order_cells(int njobs, int cells_log2 = 22)
{
    return (long long)std::max(njobs, 1) << hit_order_bits(njobs, cells_log2);
}

// shadow-ray mode of a step: packets unless the flags ask for one ray per lane
inline int shadow_packets_for(int flags) { return (flags & RP_FLAG_SHADOW_LANES) ? 0 : 1; }

struct TraceWork {
    SceneJob job0;         // the first (in single-job steps the only) job, by value
    const SceneJob *jobs;  // [njobs], device
    int njobs;
    JobState *js;          // [njobs], device
    int wave_mode;         // 1: one job, rays js[0].wave_begin + v (waves / refill)
    int plan;              // planned refill: 1 a counting pass (each path's segments only), 2 a store pass
    uint32_t *plan_seg;    // [N M] segments of candidate ray first_ray + i, or null (refill in waves)
    const RayChunk *chunks;  // [nchunks] in LPT order (wave_mode == 0)
    int nchunks;
    int chunk_rays;
    const int *src_job;    // [global sources] job of each source
    int src_base;          // global index of the group's first source
    TraceConsts k;
    const unsigned long long *seed;  // device Philox key (lo, hi words), or NULL: seed_val
    unsigned long long seed_val;
    const float4 *pos;     // sources (global index) then listeners (SceneJob::lis)
    TraceCounters *ctr;
    Hits hits;
    Records rec;
    rp_trace_stats *stats;  // aggregate statistics of the step
    uint64_t *ray_hash;     // one job: hash of primary first_ray + i at [i]
    int *status;
    // accumulation
    uint32_t *cnt, *off, *cur, *perm;  // cnt holds S T + 1 entries (it takes the segment scan)
    uint32_t *scan_part;  // tile sums of the multi-block scans (scan_parts of the longest scan)
    float *Hs, *He;  // running compensated sums [S][B][K][T] of the group
    uint32_t *segkey;     // [seg_cap] key of each segment of a heavy key (this chunk)
    float *Ss, *Se;       // [seg_cap][B K] compensated sums of those segments
    unsigned long long seg_cap;
    float *H;        // output, [global source][B][K][T]
    rp_direct *direct;  // [global sources]
    unsigned long long items_per_chunk;
    unsigned long long *rerun;  // queue of rounding-sensitive shadow items
    unsigned long long rerun_cap;
    int num_sms;
    int shadow_steps;  // node visits a shadow lane makes between refills
    HitOrder horder;   // reflections in spatial order for coherent shadow rays
    int shadow_packets;  // 1: shadow rays as warp packets, 0: one ray per lane
    Hits shits;        // point, normal, weights and ray id of the reflections in that order (shadow
                       // rays read these; the FP64 residuals stay in `hits`, found through horder.perm)
    EarlyHits er;      // early reflections (single-job steps of rp_trace_er only)
    // shadow-ray packets start at a node of the BVH around their source (src_node[global
    // source], filled by k_src_region; null: at the root); the region is the deepest
    // node on the source's side whose box is still at least region_frac of the scene
    int *src_node = nullptr;
    int *src_hint = nullptr;  // [global source * SRC_HINT_STRIDE] the latest block's hint towards it (0: none), or null
    int escalate = 0;  // walks from SHADOW_HINT_UP levels further up before the root walk
    float region_frac = 0.f;
    SpecRays spec;     // store passes of the planned refill (one job)
    unsigned long long spec_lo = 0;  // store pass: candidates from first_ray + spec_lo on are speculative
    unsigned long long rid_end = 0;  // nonzero: reflections and records of rays >= rid_end are dropped
};

void launch_setup(const TraceWork &w, int wave, cudaStream_t st);
void launch_plan_block(const TraceWork &w, unsigned long long begin, unsigned long long count, cudaStream_t st);
void launch_refill_plan(const TraceWork &w, unsigned long long candidates, cudaStream_t st);
void launch_plan_apply(const TraceWork &w, cudaStream_t st);
void launch_spec_fold(const TraceWork &w, unsigned long long count, cudaStream_t st);
void launch_paths(const TraceWork &w, int blocks, cudaStream_t st);
void launch_item_prefix(const TraceWork &w, cudaStream_t st);
void launch_hit_order(const TraceWork &w, int blocks, cudaStream_t st);
void launch_shadow(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_shadow_exact(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_direct(const TraceWork &w, cudaStream_t st);
void launch_src_region(const TraceWork &w, cudaStream_t st);
void launch_clear_counts(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_count(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_scan(const TraceWork &w, unsigned long long chunk, cudaStream_t st);
// exclusive scan; `part` (scan_parts(n) entries, or null for one block) holds tile sums
void launch_scan_u32(const uint32_t *cnt, uint32_t *off, int n, uint32_t *part, cudaStream_t st);
void launch_scatter(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_accum(const TraceWork &w, int first_chunk, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_finalize(const TraceWork &w, cudaStream_t st);
int paths_occupancy(int flags);
int shadow_occupancy(int flags);

// Host side: the launches of one trace step (one group of jobs).
typedef void (*ProfHook)(void *ctx, const char *name, int begin);

struct StepLaunch {
    TraceWork w;                      // fully populated
    unsigned long long n_rec_chunks;  // record chunks (worst case)
    int refill;                       // one job: host-synchronised refill waves
    int reset_stats;                  // zero the aggregate statistics first
    int paths_blocks, shadow_blocks, exact_blocks, flat_blocks, acc_blocks;
};
cudaError_t enqueue_step(const StepLaunch &L, cudaStream_t st, ProfHook hook, void *hook_ctx);

struct StepSizes {
    unsigned long long hit_cap, items, sph_cap, items_per_chunk, n_chunks, rec_cap, rerun_cap, keys, cells;
    unsigned long long seg_cap, seg_cells;  // segments of heavy keys a chunk can hold, and their cells
    int S;
};
// A (source, bin) with more than ACC_SEG records in a chunk is summed in segments of
// ACC_SEG records by separate warps, then the segments are combined in order.
constexpr unsigned ACC_SEG = 1024;
StepSizes step_sizes(const unsigned long long *rays, const int *sources, int njobs, int M, int B, int K, int T,
                     unsigned long long rec_budget);

struct EstimateWork {
    const float *H;
    const rp_direct *direct;
    int S, B, K, T;
    double rate, dt, tau;
    rp_reverb_params *out;
    double *state;
};
void launch_estimate(const EstimateWork &w, cudaStream_t st);

}  // namespace rp
