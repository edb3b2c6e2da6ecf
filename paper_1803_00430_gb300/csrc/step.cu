// step.cu -- the launch sequence of one trace step (one group of jobs), shared by
// rp_trace, rp_trace_noalloc and the batched entry points.
//
//   setup -> (planned refill ->) paths (-> refill waves) -> shadow-item prefix -> direct sound ->
//   per record chunk: shadow rays -> FP64 re-decisions -> count -> scan -> scatter
//   -> compensated accumulation
//   -> finalize (normalise by primaries, bin direct sound) -> status copy
//
// Everything is enqueued on one stream without host synchronisation, except the
// refill of a single-job step (the planner's passes or the next wave's size are read
// back), so a step without refill can be captured into a CUDA graph.
//
// Every stage is enqueued inside an NVTX range named after it ("rp:paths",
// "rp:shadow", ...), nested in one "rp:step" range, so that timeline and profiling
// tools can select a step or a stage (ncu --nvtx --nvtx-include "rp:step/").  Without
// a tool attached the ranges cost a few host instructions.
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

namespace rp {
namespace {

__global__ void k_copy_status(TraceWork w)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    w.stats->error = *w.status;
    unsigned long long h = 0;
    for (int j = 0; j < w.njobs; ++j) h += min(w.js[j].n_hits, w.jobs[j].hit_cap);
    w.stats->hits_stored += h;
}

// NVTX range name of a stage: "rp:" + the profiling name
inline const char *nvtx_name(const char *name)
{
    static const char *const names[][2] = {
        {"setup", "rp:setup"},         {"paths", "rp:paths"},           {"item_prefix", "rp:item_prefix"},
        {"hit_order", "rp:hit_order"}, {"direct", "rp:direct"},         {"shadow", "rp:shadow"},
        {"shadow_exact", "rp:shadow_exact"}, {"count", "rp:count"},     {"scan", "rp:scan"},
        {"scatter", "rp:scatter"},     {"accum", "rp:accum"},           {"finalize", "rp:finalize"},
        {"copy_status", "rp:copy_status"}};
    for (const auto &n : names)
        if (std::strcmp(n[0], name) == 0) return n[1];
    return "rp:stage";
}

struct Hook {
    ProfHook fn;
    void *ctx;
    const char *name;
    Hook(ProfHook f, void *c, const char *n) : fn(f), ctx(c), name(n)
    {
        nvtxRangePushA(nvtx_name(name));
        if (fn) fn(ctx, name, 1);
    }
    ~Hook()
    {
        if (fn) fn(ctx, name, 0);
        nvtxRangePop();
    }
};

// the whole step
struct StepRange {
    StepRange() { nvtxRangePushA("rp:step"); }
    ~StepRange() { nvtxRangePop(); }
};

constexpr int REFILL_BATCH = 16;  // refill waves enqueued between host checks

#define CKS(x)                                    \
    do {                                          \
        const cudaError_t e_ = (x);               \
        if (e_ != cudaSuccess) return e_;         \
    } while (0)

// Planned refill: counting passes over candidate ray ids (4 N or 4096 at first), then
// the waves' sizes.  The host reads after each pass whether more candidates are
// needed; the next pass reaches to where the segments per ray seen so far say the
// budget runs out (3 % beyond), at least to the wave that did not fit.
cudaError_t plan_refill(const TraceWork &w, int blocks, cudaStream_t st, ProfHook hook, void *hook_ctx)
{
    const unsigned long long N = w.job0.num_rays, budget = N * (unsigned long long)w.k.M;
    TraceWork wp = w;
    wp.plan = 1;
    wp.ray_hash = nullptr;
    wp.k.flags &= ~RP_FLAG_COUNT_VISITS;
    unsigned long long done = 0, cand = std::min(budget, std::max(4ull * N, 4096ull));
    for (int pass = 0; pass < 64; ++pass) {
        {
            Hook h(hook, hook_ctx, "paths");
            launch_plan_block(w, done, cand - done, st);
            launch_paths(wp, blocks, st);
        }
        done = cand;
        launch_refill_plan(w, done, st);
        unsigned long long pl[4] = {0, 0, 0, 0};  // plan_need, plan_rays, plan_waves, plan_used
        CKS(cudaMemcpyAsync(pl, &w.ctr->plan_need, sizeof(pl), cudaMemcpyDeviceToHost, st));
        CKS(cudaStreamSynchronize(st));
        const unsigned long long need = pl[0], rays = pl[1], used = pl[3];
        if (need == 0) break;
        unsigned long long next = 2 * cand;
        if (rays > 0 && used > 0 && used < budget) {
            const double per_ray = (double)used / (double)rays;
            next = (unsigned long long)(1.03 * ((double)rays + (double)(budget - used) / per_ray)) + 1024;
        }
        cand = std::min(budget, std::max(next, need));
        if (cand <= done) return cudaErrorUnknown;  // cannot happen: the waves hold at most N M rays
    }
    launch_plan_apply(w, st);
    return cudaGetLastError();
}

// Planned refill with store passes: the candidates' paths are traced once and keep
// their reflections, records and statistics.  Pass 0 takes the N primaries of the first
// wave and speculative candidates up to 4 N (at least 4096), no further than the spare
// reflection slots hold at M reflections a path.  A later pass reaches to where the
// waves are predicted to end (as in plan_refill); its last spec.cap candidates are
// speculative, the ones before them are taken as inside the waves.  When the waves
// end inside a pass, the speculative rays past them are dropped (their statistics are
// never added; their reflections and records are left out by rid_end).
// ok = false: the step has to be traced again with counting passes, because a kept
// ray lost a reflection or record for want of a slot, the waves ended before a
// candidate taken as inside them, or the source-sphere records leave the first record
// chunk too little room.
cudaError_t plan_store(const TraceWork &w, int blocks, cudaStream_t st, ProfHook hook, void *hook_ctx, bool &ok,
                       unsigned long long &K)
{
    ok = false;
    const unsigned long long N = w.job0.num_rays, M = (unsigned long long)w.k.M, budget = N * M;
    const unsigned long long spare = w.job0.hit_cap > budget ? w.job0.hit_cap - budget : 0ull;
    const size_t B = (size_t)w.k.B;
    TraceWork wp = w;
    wp.plan = 2;
    unsigned long long done = 0, lo = N;
    unsigned long long cand = std::min(std::min(budget, std::max(4ull * N, 4096ull)), N + spare / M);
    cand = std::min(cand, lo + w.spec.cap);
    for (int pass = 0; pass < 64; ++pass) {
        wp.spec_lo = lo;
        const unsigned long long nspec = cand - lo;  // cand >= lo: see below
        if (nspec) {
            CKS(cudaMemsetAsync(w.spec.late, 0, nspec * B * sizeof(double), st));
            CKS(cudaMemsetAsync(w.spec.sph, 0, nspec * sizeof(uint32_t), st));
            CKS(cudaMemsetAsync(w.spec.rerun, 0, nspec * sizeof(uint32_t), st));
        }
        {
            Hook h(hook, hook_ctx, "paths");
            launch_plan_block(w, done, cand - done, st);
            launch_paths(wp, blocks, st);
        }
        launch_refill_plan(w, cand, st);
        if (nspec) launch_spec_fold(wp, nspec, st);
        TraceCounters c;
        CKS(cudaMemcpyAsync(&c, w.ctr, sizeof(c), cudaMemcpyDeviceToHost, st));
        CKS(cudaStreamSynchronize(st));
        const unsigned long long need = c.plan_need, rays = c.plan_rays, used = c.plan_used;
        const unsigned long long taken = need ? cand : rays;  // candidates inside the waves
        if (c.store_fail && ~c.store_fail < w.job0.first_ray + taken) return cudaSuccess;
        if (need == 0) {
            if (rays < lo || c.n_records > w.rec.cap - std::min(w.rec.cap, w.items_per_chunk)) return cudaSuccess;
            K = rays;
            ok = true;
            return cudaGetLastError();
        }
        unsigned long long next = 2 * cand;
        if (rays > 0 && used > 0 && used < budget) {
            const double per_ray = (double)used / (double)rays;
            next = (unsigned long long)(1.03 * ((double)rays + (double)(budget - used) / per_ray)) + 1024;
        }
        done = cand;
        cand = std::min(budget, std::max(next, need));
        if (cand <= done) return cudaErrorUnknown;  // cannot happen: the waves hold at most N M rays
        lo = std::max(need, cand > w.spec.cap ? cand - w.spec.cap : 0ull);  // need <= cand
    }
    return cudaSuccess;  // not planned within 64 passes: counting passes instead
}

}  // namespace

cudaError_t enqueue_step(const StepLaunch &L, cudaStream_t st, ProfHook hook, void *hook_ctx)
{
    const StepRange step_range;
    TraceWork w = L.w;  // rid_end is set below once store passes have planned the refill
    const int S = w.k.S;
    CKS(cudaMemsetAsync(w.ctr, 0, sizeof(TraceCounters), st));
    CKS(cudaMemsetAsync(w.js, 0, sizeof(JobState) * (size_t)w.njobs, st));
    if (L.reset_stats) CKS(cudaMemsetAsync(w.stats, 0, sizeof(rp_trace_stats), st));
    const bool planned = L.refill && w.k.M > 0 && w.njobs == 1 && w.plan_seg;
    const bool store = planned && w.spec.cap > 0 && w.er.cap == 0 && !w.ray_hash &&
                       !(w.k.flags & (RP_FLAG_COUNT_VISITS | RP_FLAG_FP32_PATHS));
    if (store) CKS(cudaMemcpyAsync(w.spec.saved, w.stats, sizeof(rp_trace_stats), cudaMemcpyDeviceToDevice, st));
    {
        Hook h(hook, hook_ctx, "setup");
        launch_setup(w, 0, st);
    }
    bool stored = false;
    if (store) {
        unsigned long long K = 0;
        CKS(plan_store(w, L.paths_blocks, st, hook, hook_ctx, stored, K));
        if (stored) {
            launch_plan_apply(w, st);
            w.rid_end = w.job0.first_ray + K;
        } else {
            // the step again from its start, with counting passes
            CKS(cudaMemcpyAsync(w.stats, w.spec.saved, sizeof(rp_trace_stats), cudaMemcpyDeviceToDevice, st));
            CKS(cudaMemsetAsync(w.ctr, 0, sizeof(TraceCounters), st));
            CKS(cudaMemsetAsync(w.js, 0, sizeof(JobState) * (size_t)w.njobs, st));
            Hook h(hook, hook_ctx, "setup");
            launch_setup(w, 0, st);
        }
    }
    if (planned && !stored) CKS(plan_refill(w, L.paths_blocks, st, hook, hook_ctx));
    if (w.k.M > 0 && !stored) {
        Hook h(hook, hook_ctx, "paths");
        launch_paths(w, L.paths_blocks, st);
    }
    if (L.refill && w.k.M > 0 && w.njobs == 1 && !planned) {
        // Refill waves go out REFILL_BATCH at a time with no host synchronisation in
        // between: a wave whose budget is spent has no rays, its setup leaves the state
        // as it is and its paths launch returns at once.  The host reads the last wave's
        // size after each batch and stops once it is zero.
        for (int wave = 1; wave < 4096; wave += REFILL_BATCH) {
            for (int k = 0; k < REFILL_BATCH; ++k) {
                {
                    Hook h(hook, hook_ctx, "setup");
                    launch_setup(w, wave + k, st);
                }
                Hook h(hook, hook_ctx, "paths");
                launch_paths(w, L.paths_blocks, st);
            }
            unsigned long long cnt = 0;
            CKS(cudaMemcpyAsync(&cnt, &w.js[0].wave_count, sizeof(cnt), cudaMemcpyDeviceToHost, st));
            CKS(cudaStreamSynchronize(st));
            if (cnt == 0) break;
        }
    }
    {
        Hook h(hook, hook_ctx, "item_prefix");
        launch_item_prefix(w, st);
    }
    if (S > 0 && w.k.M > 0) {
        Hook h(hook, hook_ctx, "hit_order");
        launch_hit_order(w, L.flat_blocks, st);
    }
    {
        Hook h(hook, hook_ctx, "direct");
        launch_direct(w, st);
        launch_src_region(w, st);
    }
    for (unsigned long long ch = 0; ch < L.n_rec_chunks && S > 0; ++ch) {
        if (ch > 0) CKS(cudaMemsetAsync(&w.ctr->n_records, 0, sizeof(unsigned long long), st));
        CKS(cudaMemsetAsync(&w.ctr->next_item, 0, 2 * sizeof(unsigned long long), st));  // + n_rerun
        if (w.k.M > 0) {
            {
                Hook h(hook, hook_ctx, "shadow");
                launch_shadow(w, ch, L.shadow_blocks, st);
            }
            Hook h(hook, hook_ctx, "shadow_exact");
            launch_shadow_exact(w, ch, L.exact_blocks, st);
        }
        {
            Hook h(hook, hook_ctx, "count");
            launch_clear_counts(w, ch, L.flat_blocks, st);
            launch_count(w, ch, L.flat_blocks, st);
        }
        {
            Hook h(hook, hook_ctx, "scan");
            launch_scan(w, ch, st);
        }
        {
            Hook h(hook, hook_ctx, "scatter");
            launch_scatter(w, ch, L.flat_blocks, st);
        }
        {
            Hook h(hook, hook_ctx, "accum");
            launch_accum(w, ch == 0 ? 1 : 0, ch, L.acc_blocks, st);
        }
    }
    if (S > 0) {
        Hook h(hook, hook_ctx, "finalize");
        launch_finalize(w, st);
    }
    {
        Hook h(hook, hook_ctx, "copy_status");
        k_copy_status<<<1, 1, 0, st>>>(w);
    }
    return cudaGetLastError();
}

// Worst-case sizes of a group: reflections, shadow items and record chunks.
StepSizes step_sizes(const unsigned long long *rays, const int *sources, int njobs, int M, int B, int K, int T,
                     unsigned long long rec_budget)
{
    StepSizes z;
    z.hit_cap = 0;
    z.items = 0;
    z.S = 0;
    for (int j = 0; j < njobs; ++j) {
        const unsigned long long h = rays[j] * (unsigned long long)std::max(M, 0);
        z.hit_cap += h;
        z.items += shadow_items(h, sources[j]);
        z.S += sources[j];
    }
    z.hit_cap = std::max(1ull, z.hit_cap);
    z.sph_cap = z.hit_cap / 2 + 4096;
    const unsigned long long room = rec_budget > z.sph_cap + 1 ? rec_budget - z.sph_cap : 1ull << 20;
    // a multiple of a warp's block of tiles, so that a block's runs stay whole (a multiple
    // of 32 when the room is smaller: a warp's 32 consecutive items stay one run)
    const unsigned long long blk = 32ull * SHADOW_TILE_GROUP, fit = std::min(std::max(z.items, 1ull), room);
    z.items_per_chunk = fit >= blk ? fit / blk * blk : std::max(32ull, fit / 32ull * 32ull);
    z.n_chunks = (std::max(z.items, 1ull) + z.items_per_chunk - 1) / z.items_per_chunk;
    z.rec_cap = z.sph_cap + z.items_per_chunk;
    z.rerun_cap = z.rec_cap / 8 + 4096;
    z.keys = (unsigned long long)z.S * T;
    z.cells = z.keys * B * K;
    // a heavy key (more than ACC_SEG records) has at most 2 c / ACC_SEG segments
    z.seg_cap = 2 * z.rec_cap / ACC_SEG + 2;
    z.seg_cells = z.seg_cap * B * K;
    return z;
}

}  // namespace rp
