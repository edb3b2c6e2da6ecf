// internal.cuh -- data structures and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

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
    float tmin;     // self-intersection guard used by FP32 queries
    double tmin_d;  // the same guard for FP64 re-decisions
};

// Counters and accumulators of one trace step (device memory, zeroed per step).
struct TraceCounters {
    unsigned long long next_ray;     // primaries handed out in the current wave
    unsigned long long wave_begin;   // first ray id of the current wave
    unsigned long long wave_count;   // primaries in the current wave
    unsigned long long n_hits;       // stored reflections (next-event work)
    unsigned long long n_records;    // contribution records in the current chunk
    unsigned long long n_sphere;     // records written by the path kernel
    unsigned long long next_item;    // shadow work fetched in the current chunk
    unsigned long long n_rerun;      // shadow items queued for an FP64 decision (current chunk)
};

// Contribution records: key = source * T + bin, ray id, e[B] (row of B floats).
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
    float *ws;      // [b * cap + j] path weight after absorption times s_b
    uint32_t *rid;  // primary ray id
    unsigned long long cap;
};

struct TraceConsts {
    int S, B, K, T, M, min_order, sh_order;
    float rate, c, rs;
    uint32_t scene_id, key0, key1;
    uint64_t num_rays, first_ray;
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
};

// Builds the BVH; all temporaries are allocated and freed inside.  Returns a
// cudaError_t; device-detected input errors go to *status.
cudaError_t build_bvh(const BvhBuildArgs &a, BvhOut &out, int *d_status, cudaStream_t st);

struct TraceWork {
    SceneView sc;
    TraceConsts k;
    const float4 *src;   // [S + 1] sources then the listener, (x, y, z, 0), device
    TraceCounters *ctr;
    Hits hits;
    Records rec;
    rp_trace_stats *stats;  // device accumulators
    uint64_t *ray_hash;
    int *status;
    // accumulation
    uint32_t *cnt, *off, *cur, *perm;
    float *Hs, *He;  // running compensated sums [S][B][K][T]
    float *H;        // output
    rp_direct *direct;
    unsigned long long hits_per_chunk;
    unsigned long long *rerun;  // queue of rounding-sensitive shadow items
    unsigned long long rerun_cap;
    int num_sms;
};

void launch_wave_setup(const TraceWork &w, int wave, cudaStream_t st);
void launch_paths(const TraceWork &w, int blocks, cudaStream_t st);
void launch_shadow(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_shadow_exact(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st);
void launch_direct(const TraceWork &w, cudaStream_t st);
void launch_count(const TraceWork &w, int blocks, cudaStream_t st);
void launch_scan(const TraceWork &w, cudaStream_t st);
void launch_scatter(const TraceWork &w, int blocks, cudaStream_t st);
void launch_accum(const TraceWork &w, int first_chunk, int blocks, cudaStream_t st);
void launch_finalize(const TraceWork &w, cudaStream_t st);
int paths_occupancy(int flags);
int shadow_occupancy(int flags);

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
