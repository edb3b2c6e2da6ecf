// handles.cuh -- the library's opaque handle types (rp_ctx, rp_scene), shared by the
// translation units that implement the C ABI.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "internal.cuh"

namespace rp {

// Refill budgets N M up to this many segments are planned (one u32 per candidate ray);
// larger ones run as host-checked waves.
constexpr unsigned long long PLAN_MAX_RAYS = 1ull << 28;

// Records kept in device memory at once (one chunk of next-event work plus the
// records of source-sphere hits): 2^30, 44 bytes each at 8 bands with the sort index
// (47 GB at most; a problem takes only what its worst case needs).  Record chunks
// are sized for the worst case and every chunk launches its kernels, so fewer,
// larger chunks save launches on problems whose worst case is far above their work.
constexpr unsigned long long REC_BUDGET = 1ull << 30;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct ProfPair {
    const char *name;
    cudaEvent_t a, b;
};

}  // namespace rp

using rp::Buf;
using rp::ProfPair;

struct rp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int *d_status = nullptr;
    int paths_blocks = 0, shadow_blocks = 0;
    int shadow_steps = 8;  // node visits a shadow-ray lane makes between refills (one-ray-per-lane mode)
    float region_frac = 1.0f / 32;  // a source's region: at least this share of the scene's extent
    int escalate = 2;  // shadow packets: walks from further up before the root walk
    rp_debug_limits dbg = {0, 0, 0ull, 0ull};  // rp_set_debug_limits (all zero: the normal limits)
    unsigned long long ws_gen = 0;  // bumped whenever a workspace buffer is reallocated
    // workspace
    //   stored reflections (hit_*), their cell-ordered copy (shit_*) and order (hord_*),
    //   contribution records and their counting sort, running histogram sums, positions,
    //   counters, statistics, the host-buffer update's outputs, job tables, the refill
    //   planner's segment counts (plan_seg) and speculative rays (spec)
    Buf hit_p, hit_plo, hit_n, hit_ws, hit_rid, shit_p, shit_n, shit_ws, shit_rid, hord_cell, hord_perm, hord_cnt,
        rec_key, rec_rid, rec_e, perm, rerun, cnt, off, cur, scan_part, Hs, He, src, ctr, stats, H, direct, params,
        state, jobs, js, chunks, src_job, src_node, plan_seg, spec, segkey, seg_s, seg_e;
    Buf rv_raw, rv_bands, rv_comb, rv_ap, rv_phi;  // reverberator rendering: band signals, comb and all-pass
                                                  // signals, the crossover's chunk transition
    // profiling
    bool prof = false;
    std::vector<ProfPair> pending;
    std::vector<ProfPair> open_events;
    std::vector<cudaEvent_t> free_events;
    std::map<std::string, std::pair<unsigned long long, double>> totals;
};

struct rp_scene {
    rp_ctx *ctx = nullptr;
    int num_tris = 0, num_nodes = 0, num_mats = 0, B = 0, max_depth = 0, num_verts = 0;
    float tmin = 0.f, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, build_ms = 0.f, refit_ms = 0.f;
    float ray_eps = 0.f;             // the mesh's ray_epsilon (0: t_min follows the bounds)
    int32_t *vidx = nullptr;         // [num_tris][3] vertex indices (input order), for refits
    int *pleaf = nullptr, *pint = nullptr;  // parents of leaves and internal nodes (refits)
    int *anc = nullptr;                     // ancestors of the leaves (shadow-ray hints)
    int *up = nullptr;                      // ancestors of the internal nodes (shadow-ray hints)
    double tmin_d = 0.0;
    float4 *nodes = nullptr, *tris = nullptr;
    float *alpha = nullptr, *scat = nullptr, *wdiff = nullptr, *wspec = nullptr;
    uint32_t *thr = nullptr;
};

namespace rp {
// The trace step of rp_trace (api.cu), optionally keeping the early reflections for
// rp_trace_er; *work_out (if given) receives the step's bindings.
int trace_enqueue(rp_scene *sc, const rp_trace_params *p, const float *listener, const float *sources, int32_t S,
                  float *H, rp_direct *direct, rp_trace_stats *stats, uint64_t *ray_hash, const EarlyHits *early,
                  TraceWork *work_out);
}  // namespace rp

// the device view of a scene that a trace step uses
inline rp::SceneView make_view(const rp_scene *sc)
{
    rp::SceneView v = {sc->nodes, sc->tris, sc->alpha, sc->scat, sc->wdiff, sc->wspec, sc->thr, sc->num_tris,
                       sc->num_nodes, sc->B, rp::ITER_CAP_MULT * sc->num_nodes + 64, sc->tmin, sc->tmin_d,
                       {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    for (int a = 0; a < 3; ++a) {
        v.lo[a] = sc->lo[a];
        v.ext[a] = sc->hi[a] - sc->lo[a];
    }
    v.anc = sc->anc;
    v.up = sc->up;
    return v;
}

// Kernel timing while profiling is enabled (rp_profile_enable): events recorded on the
// context stream around a launch; rp_profile_read adds them up per name.
inline cudaEvent_t get_event(rp_ctx *c)
{
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    rp_ctx *c;
    const char *name;
    cudaEvent_t a = nullptr;
    ProfScope(rp_ctx *c_, const char *n) : c(c_), name(n)
    {
        if (c->prof) {
            a = get_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~ProfScope()
    {
        if (c->prof && a) {
            cudaEvent_t b = get_event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({name, a, b});
        }
    }
};
