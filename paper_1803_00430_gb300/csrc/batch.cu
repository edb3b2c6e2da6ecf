// batch.cu -- many independent scenes (each with its own sources, listener and ray
// budget) traced and estimated in the same persistent launches, captured once in a
// CUDA graph and replayed per update, with an autotuner for the launch shapes.
//
// A batch holds a device table of jobs (scene geometry, rays, sources, listener,
// region of the reflection buffer).  Jobs are grouped so that one group's stored
// reflections fit the workspace budget; each group is one step (enqueue_step):
// one paths launch over all its jobs (primaries handed out in chunks, chunks of the
// costliest scenes first -- longest-processing-time order), one shadow-ray launch
// over all its (reflection, source) items, one accumulation over all its
// (source, bin) keys.  The estimator then runs over every source of the batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "handles.cuh"

using namespace rp;

namespace {

// reflections stored at once by one group (84 B each at 8 bands)
constexpr unsigned long long HIT_BUDGET = 1ull << 27;

}  // namespace

struct rp_batch {
    rp_ctx *ctx = nullptr;
    cudaStream_t own_stream = nullptr;  // used when the context stream is the legacy default
    int n = 0, S_total = 0, B = 0, K = 0, T = 0;
    rp_trace_params common;
    rp_estimate_params est;
    float *H = nullptr;
    rp_direct *direct = nullptr;
    rp_reverb_params *params = nullptr;
    rp_trace_stats *stats = nullptr;
    std::vector<SceneJob> h_jobs;
    std::vector<int> h_src_job;
    std::vector<int> tri_count;
    SceneJob *d_jobs = nullptr;
    RayChunk *d_chunks = nullptr;
    int *d_src_job = nullptr;
    int *d_src_node = nullptr;  // start node of each source's shadow-ray packets, then their latest hints
    float4 *d_pos = nullptr;
    unsigned long long *d_seed = nullptr;
    unsigned long long *h_seed = nullptr;  // pinned
    struct Group {
        int job_begin, job_end, src_begin, src_count;
        StepSizes z;
        int chunk_begin, nchunks;
    };
    std::vector<Group> groups;
    StepSizes zmax;
    int max_jobs = 0;
    int max_chunks = 0;
    rp_batch_tuning tuning;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    unsigned long long graph_gen = ~0ull;
};

namespace {

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return RP_OK;
    if (e == cudaErrorMemoryAllocation) return RP_ERR_OOM;
    return RP_ERR_CUDA;
}

#define CKB(x)                                     \
    do {                                           \
        const cudaError_t e_ = (x);                \
        if (e_ != cudaSuccess) return cuda_rc(e_); \
    } while (0)

cudaStream_t batch_stream(const rp_batch *b) { return b->ctx->stream ? b->ctx->stream : b->own_stream; }

void drop_graph(rp_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->graph_gen = ~0ull;
}

// chunk tables of every group: chunk_rays primaries per chunk, chunks of the jobs
// with the most triangles first (longest-processing-time order)
int build_chunks(rp_batch *b)
{
    std::vector<RayChunk> all;
    const int cr = b->tuning.chunk_rays;
    b->max_chunks = 1;
    for (auto &g : b->groups) {
        std::vector<int> order;
        for (int j = g.job_begin; j < g.job_end; ++j) order.push_back(j);
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return b->tri_count[x] > b->tri_count[y]; });
        g.chunk_begin = (int)all.size();
        for (int j : order) {
            const SceneJob &J = b->h_jobs[j];
            for (unsigned long long r = 0; r < J.num_rays; r += (unsigned long long)cr) {
                RayChunk c;
                c.job = j - g.job_begin;
                c.count = (int)std::min<unsigned long long>((unsigned long long)cr, J.num_rays - r);
                c.start = J.first_ray + r;
                all.push_back(c);
            }
        }
        g.nchunks = (int)all.size() - g.chunk_begin;
        b->max_chunks = std::max(b->max_chunks, g.nchunks);
    }
    if (b->d_chunks) cudaFree(b->d_chunks);
    b->d_chunks = nullptr;
    CKB(cudaMalloc(&b->d_chunks, sizeof(RayChunk) * std::max<size_t>(all.size(), 1)));
    CKB(cudaMemcpy(b->d_chunks, all.data(), sizeof(RayChunk) * all.size(), cudaMemcpyHostToDevice));
    return RP_OK;
}

int grow(rp_ctx *c, Buf &buf, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (buf.bytes >= bytes) return RP_OK;
    CKB(cudaStreamSynchronize(c->stream));
    if (buf.p) cudaFree(buf.p);
    buf.p = nullptr;
    buf.bytes = 0;
    CKB(cudaMalloc(&buf.p, bytes));
    buf.bytes = bytes;
    c->ws_gen++;
    return RP_OK;
}

int reserve_batch(rp_batch *b)
{
    rp_ctx *c = b->ctx;
    const StepSizes &z = b->zmax;
    const int B = b->B;
    int r;
    if ((r = grow(c, c->hit_p, z.hit_cap * sizeof(float4)))) return r;
    if ((r = grow(c, c->hit_plo, z.hit_cap * sizeof(float4)))) return r;
    if ((r = grow(c, c->hit_n, z.hit_cap * sizeof(float4)))) return r;
    if ((r = grow(c, c->hit_ws, z.hit_cap * B * sizeof(float)))) return r;
    if ((r = grow(c, c->hit_rid, z.hit_cap * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->hord_cell, z.hit_cap * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->shit_p, z.hit_cap * sizeof(float4)))) return r;
    if ((r = grow(c, c->hord_perm, z.hit_cap * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->shit_n, z.hit_cap * sizeof(float4)))) return r;
    if ((r = grow(c, c->shit_ws, z.hit_cap * B * sizeof(float)))) return r;
    if ((r = grow(c, c->shit_rid, z.hit_cap * sizeof(uint32_t)))) return r;
    const long long cells = std::max(1ll << 22, 8ll * b->max_jobs) + 1;  // >= hit_order_cells of any group
    if ((r = grow(c, c->hord_cnt, (size_t)cells * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->rec_key, z.rec_cap * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->rec_rid, z.rec_cap * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->rec_e, z.rec_cap * B * sizeof(float)))) return r;
    if ((r = grow(c, c->perm, z.rec_cap * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->rerun, z.rerun_cap * sizeof(unsigned long long)))) return r;
    if ((r = grow(c, c->cnt, (z.keys + 1) * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->cur, z.keys * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->segkey, z.seg_cap * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->seg_s, z.seg_cells * sizeof(float)))) return r;
    if ((r = grow(c, c->seg_e, z.seg_cells * sizeof(float)))) return r;
    if ((r = grow(c, c->off, (z.keys + 1) * sizeof(uint32_t)))) return r;
    if ((r = grow(c, c->scan_part, scan_parts(std::max<unsigned long long>(z.keys, cells)) * sizeof(uint32_t))))
        return r;
    if ((r = grow(c, c->Hs, z.cells * sizeof(float)))) return r;
    if ((r = grow(c, c->He, z.cells * sizeof(float)))) return r;
    if ((r = grow(c, c->js, (size_t)b->max_jobs * sizeof(JobState)))) return r;
    if ((r = grow(c, c->ctr, sizeof(TraceCounters)))) return r;
    if ((r = grow(c, c->stats, sizeof(rp_trace_stats)))) return r;
    return RP_OK;
}

StepLaunch group_launch(const rp_batch *b, const rp_batch::Group &g)
{
    rp_ctx *c = b->ctx;
    StepLaunch L;
    TraceWork &w = L.w;
    w.ctr = (TraceCounters *)c->ctr.p;
    w.hits = {(float4 *)c->hit_p.p, (float4 *)c->hit_plo.p, (float4 *)c->hit_n.p, (float *)c->hit_ws.p,
              (uint32_t *)c->hit_rid.p, b->zmax.hit_cap};
    w.rec = {(uint32_t *)c->rec_key.p, (uint32_t *)c->rec_rid.p, (float *)c->rec_e.p, g.z.rec_cap};
    w.stats = (rp_trace_stats *)c->stats.p;
    w.status = c->d_status;
    w.cnt = (uint32_t *)c->cnt.p;
    w.off = (uint32_t *)c->off.p;
    w.scan_part = (uint32_t *)c->scan_part.p;
    w.cur = (uint32_t *)c->cur.p;
    w.perm = (uint32_t *)c->perm.p;
    w.Hs = (float *)c->Hs.p;
    w.He = (float *)c->He.p;
    w.segkey = (uint32_t *)c->segkey.p;
    w.Ss = (float *)c->seg_s.p;
    w.Se = (float *)c->seg_e.p;
    w.seg_cap = g.z.seg_cap;
    w.items_per_chunk = g.z.items_per_chunk;
    w.rerun = (unsigned long long *)c->rerun.p;
    w.rerun_cap = g.z.rerun_cap;
    w.num_sms = c->num_sms;
    w.job0 = b->h_jobs[g.job_begin];
    w.jobs = b->d_jobs + g.job_begin;
    w.njobs = g.job_end - g.job_begin;
    w.shits = {(float4 *)c->shit_p.p, nullptr, (float4 *)c->shit_n.p, (float *)c->shit_ws.p,
               (uint32_t *)c->shit_rid.p, b->zmax.hit_cap};
    w.horder = {(uint32_t *)c->hord_cell.p, (uint32_t *)c->hord_perm.p, (uint32_t *)c->hord_cnt.p,
                hit_order_bits(w.njobs), (int)hit_order_cells(w.njobs)};
    w.js = (JobState *)c->js.p;
    w.wave_mode = 0;
    w.plan = 0;
    w.plan_seg = nullptr;
    w.chunks = b->d_chunks + g.chunk_begin;
    w.nchunks = g.nchunks;
    w.chunk_rays = b->tuning.chunk_rays;
    w.src_job = b->d_src_job;
    w.src_node = b->d_src_node;
    w.src_hint = b->d_src_node + b->h_src_job.size();
    w.region_frac = c->region_frac;
    w.escalate = c->escalate;
    w.src_base = g.src_begin;
    w.k.S = g.src_count;
    w.k.B = b->B;
    w.k.K = b->K;
    w.k.T = b->T;
    w.k.M = b->common.max_order;
    w.k.min_order = b->common.min_order;
    w.k.sh_order = b->common.sh_order;
    w.k.rate = b->common.ir_rate_hz;
    w.k.c = b->common.speed_of_sound;
    w.k.rs = b->common.source_radius;
    w.k.flags = b->common.flags & ~(RP_FLAG_RAY_HASH | RP_FLAG_DEVICE_POSITIONS);
    w.seed = b->d_seed;
    w.seed_val = 0;
    w.pos = b->d_pos;
    w.ray_hash = nullptr;
    w.H = b->H;
    w.direct = b->direct;
    w.shadow_steps = b->tuning.shadow_steps;
    {
        const int mode = b->tuning.shadow_mode;
        w.shadow_packets = mode == 1 ? 1 : mode == 2 ? 0 : shadow_packets_for(b->common.flags);
    }
    L.n_rec_chunks = g.z.n_chunks;
    L.refill = 0;
    L.reset_stats = &g == &b->groups.front();
    L.paths_blocks = c->num_sms * b->tuning.paths_blocks_per_sm;
    L.shadow_blocks = c->num_sms * b->tuning.shadow_blocks_per_sm;
    L.exact_blocks = c->num_sms * 2;
    L.flat_blocks = c->num_sms * 8;
    L.acc_blocks = (int)std::max(1ll, std::min<long long>(((long long)g.z.keys + 7) / 8, (long long)c->num_sms * 8));
    return L;
}

// every launch of one batched update (all groups, then the estimator)
int enqueue_all(rp_batch *b, cudaStream_t st, bool profile)
{
    for (const auto &g : b->groups) {
        const StepLaunch L = group_launch(b, g);
        CKB(enqueue_step(L, st, nullptr, nullptr));
    }
    (void)profile;
    if (b->params && b->S_total > 0) {
        EstimateWork ew{b->H, b->direct, b->S_total, b->B, b->K, b->T, b->est.ir_rate_hz, b->est.dt_update,
                        b->est.tau, b->params, nullptr};
        launch_estimate(ew, st);
    }
    if (b->stats)
        CKB(cudaMemcpyAsync(b->stats, b->ctx->stats.p, sizeof(rp_trace_stats), cudaMemcpyDeviceToDevice, st));
    return cuda_rc(cudaGetLastError());
}

int run_once(rp_batch *b, unsigned long long seed, int use_graph)
{
    rp_ctx *c = b->ctx;
    cudaStream_t st = batch_stream(b);
    int r;
    if ((r = reserve_batch(b))) return r;  // no-op unless another call shrank nothing... grows only
    *b->h_seed = seed;
    CKB(cudaMemcpyAsync(b->d_seed, b->h_seed, sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    if (use_graph) {
        if (!b->gexec || b->graph_gen != c->ws_gen) {
            drop_graph(b);
            CKB(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue_all(b, st, false);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            CKB(e);
            b->graph = g;
            CKB(cudaGraphInstantiate(&b->gexec, g, 0));
            b->graph_gen = c->ws_gen;
        }
        CKB(cudaGraphLaunch(b->gexec, st));
    } else {
        if ((r = enqueue_all(b, st, true))) return r;
    }
    if (st != c->stream) {
        // the context stream (the legacy default) waits for the batch stream
        cudaEvent_t ev;
        CKB(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, st);
        cudaStreamWaitEvent(c->stream, ev, 0);
        cudaEventDestroy(ev);
    }
    return RP_OK;
}

std::string tuning_key(const rp_batch *b)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, b->ctx->device);
    unsigned long long rays = 0, tris = 0;
    for (size_t j = 0; j < b->h_jobs.size(); ++j) {
        rays += b->h_jobs[j].num_rays;
        tris += (unsigned long long)b->tri_count[j];
    }
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|sm%d|n%d|src%d|rays%llu|tris%llu|M%d|B%d|K%d|T%d|f%d", prop.name,
             prop.multiProcessorCount, b->n, b->S_total, rays, tris, b->common.max_order, b->B, b->K, b->T,
             b->common.flags & RP_FLAG_FP32_PATHS);
    std::string s(buf);
    for (auto &ch : s)
        if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
    return s;
}

bool cache_lookup(const char *path, const std::string &key, rp_batch_tuning &t, double &ms)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[600];
        rp_batch_tuning x;
        double m;
        if (sscanf(line, "%599s %d %d %d %d %d %lf", k, &x.chunk_rays, &x.shadow_steps, &x.paths_blocks_per_sm,
                   &x.shadow_blocks_per_sm, &x.shadow_mode, &m) == 7 &&
            key == k) {
            t = x;
            ms = m;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const rp_batch_tuning &t, double ms)
{
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %.6f\n", key.c_str(), t.chunk_rays, t.shadow_steps, t.paths_blocks_per_sm,
            t.shadow_blocks_per_sm, t.shadow_mode, ms);
    fclose(f);
}

bool tuning_valid(const rp_batch *b, const rp_batch_tuning &t)
{
    const int pocc = paths_occupancy(b->common.flags), socc = shadow_occupancy(b->common.flags);
    return t.chunk_rays >= 32 && t.chunk_rays <= 65536 && t.shadow_steps >= 1 && t.shadow_steps <= 64 &&
           t.paths_blocks_per_sm >= 1 && t.paths_blocks_per_sm <= pocc && t.shadow_blocks_per_sm >= 1 &&
           t.shadow_blocks_per_sm <= socc && t.shadow_mode >= 0 && t.shadow_mode <= 2;
}

}  // namespace

extern "C" {

int rp_batch_create(rp_ctx *c, const rp_batch_item *items, int32_t n, const rp_trace_params *p,
                    const rp_estimate_params *est, float *H, rp_direct *direct, rp_reverb_params *params,
                    rp_trace_stats *stats, rp_batch **out)
{
    if (!c || !items || n <= 0 || !p || !H || !direct || !out || (params && !est)) return RP_ERR_INVALID_ARG;
    *out = nullptr;
    if (p->budget_refill || (p->flags & (RP_FLAG_RAY_HASH | RP_FLAG_DEVICE_POSITIONS))) return RP_ERR_INVALID_ARG;
    if ((p->flags & RP_FLAG_SHADOW_PACKETS) && (p->flags & RP_FLAG_SHADOW_LANES)) return RP_ERR_INVALID_ARG;
    if (p->max_order < 0 || p->sh_order < 0 || p->sh_order > RP_MAX_SH_ORDER || p->num_bins < 1 ||
        p->min_order < 0 || !(p->ir_rate_hz > 0.f) || !(p->speed_of_sound > 0.f) || !(p->source_radius > 0.f))
        return RP_ERR_INVALID_ARG;
    int B = -1;
    long long S_total = 0;
    for (int i = 0; i < n; ++i) {
        const rp_batch_item &it = items[i];
        if (!it.scene || it.scene->ctx != c || it.num_sources < 0 || it.num_sources > RP_MAX_SOURCES ||
            !it.listener || (it.num_sources > 0 && !it.sources) || it.num_rays > 0xffffffffull ||
            it.first_ray > 0x100000000ull - it.num_rays)  // 32-bit ray ids, no wrap
            return RP_ERR_INVALID_ARG;
        if (B < 0) B = it.scene->B;
        if (it.scene->B != B) return RP_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(it.listener[k])) return RP_ERR_NAN_INPUT;
        for (long long k = 0; k < 3ll * it.num_sources; ++k)
            if (!std::isfinite(it.sources[k])) return RP_ERR_NAN_INPUT;
        S_total += it.num_sources;
    }
    if (S_total * (long long)p->num_bins >= (1ll << 31)) return RP_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return RP_ERR_CUDA;
    rp_batch *b = new (std::nothrow) rp_batch();
    if (!b) return RP_ERR_OOM;
    b->ctx = c;
    b->n = n;
    b->S_total = (int)S_total;
    b->B = B;
    b->K = (p->sh_order + 1) * (p->sh_order + 1);
    b->T = p->num_bins;
    b->common = *p;
    if (est) b->est = *est;
    b->H = H;
    b->direct = direct;
    b->params = params;
    b->stats = stats;
    b->tuning = {256, c->shadow_steps, paths_occupancy(p->flags), shadow_occupancy(p->flags), 0};
    const int M = p->max_order;
    // jobs, positions (all sources, then one listener per job), source -> job
    std::vector<float4> pos((size_t)S_total + n);
    b->h_src_job.assign((size_t)std::max<long long>(S_total, 1), 0);
    int src = 0;
    for (int i = 0; i < n; ++i) {
        const rp_batch_item &it = items[i];
        SceneJob J;
        const rp_scene *sc = it.scene;
        J.sc = make_view(sc);
        J.first_ray = it.first_ray;
        J.num_rays = it.num_rays;
        J.hit_off = 0;
        J.hit_cap = it.num_rays * (unsigned long long)std::max(M, 0);
        J.scene_id = it.scene_id;
        J.S = it.num_sources;
        J.src_off = src;
        J.lis = (int)S_total + i;
        for (int s = 0; s < it.num_sources; ++s)
            pos[src + s] = make_float4(it.sources[3 * s], it.sources[3 * s + 1], it.sources[3 * s + 2], 0.f);
        pos[S_total + i] = make_float4(it.listener[0], it.listener[1], it.listener[2], 0.f);
        src += it.num_sources;
        b->h_jobs.push_back(J);
        b->tri_count.push_back(sc->num_tris);
    }
    // groups: consecutive jobs whose reflections fit the budget; job-local indices.
    // RP_BATCH_HIT_BUDGET (reflections) lowers the budget, e.g. to exercise several groups.
    unsigned long long hit_budget = HIT_BUDGET;
    if (const char *env = getenv("RP_BATCH_HIT_BUDGET")) {
        const unsigned long long v = strtoull(env, nullptr, 10);
        if (v > 0) hit_budget = std::min(v, HIT_BUDGET);
    }
    int j = 0;
    memset(&b->zmax, 0, sizeof(b->zmax));
    while (j < n) {
        rp_batch::Group g;
        g.job_begin = j;
        unsigned long long hits = 0;
        while (j < n && (j == g.job_begin || hits + b->h_jobs[j].hit_cap <= hit_budget)) {
            b->h_jobs[j].hit_off = hits;
            hits += b->h_jobs[j].hit_cap;
            ++j;
        }
        g.job_end = j;
        g.src_begin = b->h_jobs[g.job_begin].src_off;
        g.src_count = 0;
        std::vector<unsigned long long> rays;
        std::vector<int> srcs;
        for (int q = g.job_begin; q < g.job_end; ++q) {
            g.src_count += b->h_jobs[q].S;
            rays.push_back(b->h_jobs[q].num_rays);
            srcs.push_back(b->h_jobs[q].S);
            for (int s = 0; s < b->h_jobs[q].S; ++s) b->h_src_job[b->h_jobs[q].src_off + s] = q - g.job_begin;
        }
        g.z = step_sizes(rays.data(), srcs.data(), g.job_end - g.job_begin, M, B, b->K, b->T, REC_BUDGET);
        StepSizes &zm = b->zmax;
        zm.hit_cap = std::max(zm.hit_cap, g.z.hit_cap);
        zm.rec_cap = std::max(zm.rec_cap, g.z.rec_cap);
        zm.rerun_cap = std::max(zm.rerun_cap, g.z.rerun_cap);
        zm.keys = std::max(zm.keys, g.z.keys);
        zm.cells = std::max(zm.cells, g.z.cells);
        zm.seg_cap = std::max(zm.seg_cap, g.z.seg_cap);
        zm.seg_cells = std::max(zm.seg_cells, g.z.seg_cells);
        b->max_jobs = std::max(b->max_jobs, g.job_end - g.job_begin);
        b->groups.push_back(g);
    }
    int rc = RP_OK;
    cudaError_t e;
    if (!c->stream && (e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        rc = cuda_rc(e);
        goto fail;
    }
    if ((e = cudaMalloc(&b->d_jobs, sizeof(SceneJob) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_src_job, sizeof(int) * b->h_src_job.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_src_node, (1 + SRC_HINT_STRIDE) * sizeof(int) * b->h_src_job.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_pos, sizeof(float4) * pos.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_seed, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_seed, sizeof(unsigned long long))) != cudaSuccess) {
        rc = cuda_rc(e);
        goto fail;
    }
    if ((e = cudaMemcpy(b->d_jobs, b->h_jobs.data(), sizeof(SceneJob) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_src_job, b->h_src_job.data(), sizeof(int) * b->h_src_job.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_pos, pos.data(), sizeof(float4) * pos.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
        rc = cuda_rc(e);
        goto fail;
    }
    if ((rc = build_chunks(b))) goto fail;
    if ((rc = reserve_batch(b))) goto fail;
    *out = b;
    return RP_OK;
fail:
    rp_batch_destroy(b);
    return rc;
}

int rp_batch_destroy(rp_batch *b)
{
    if (!b) return RP_ERR_INVALID_ARG;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(batch_stream(b));
    drop_graph(b);
    cudaFree(b->d_jobs);
    cudaFree(b->d_chunks);
    cudaFree(b->d_src_job);
    cudaFree(b->d_src_node);
    cudaFree(b->d_pos);
    cudaFree(b->d_seed);
    if (b->h_seed) cudaFreeHost(b->h_seed);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return RP_OK;
}

int rp_batch_run(rp_batch *b, uint64_t seed, int use_graph)
{
    if (!b) return RP_ERR_INVALID_ARG;
    if (cudaSetDevice(b->ctx->device) != cudaSuccess) return RP_ERR_CUDA;
    return run_once(b, seed, use_graph);
}

int rp_batch_set_tuning(rp_batch *b, const rp_batch_tuning *t)
{
    if (!b || !t || !tuning_valid(b, *t)) return RP_ERR_INVALID_ARG;
    if (cudaSetDevice(b->ctx->device) != cudaSuccess) return RP_ERR_CUDA;
    cudaStreamSynchronize(batch_stream(b));
    const bool rechunk = t->chunk_rays != b->tuning.chunk_rays;
    b->tuning = *t;
    drop_graph(b);
    return rechunk ? build_chunks(b) : RP_OK;
}

int rp_batch_get_tuning(const rp_batch *b, rp_batch_tuning *t)
{
    if (!b || !t) return RP_ERR_INVALID_ARG;
    *t = b->tuning;
    return RP_OK;
}

int rp_batch_info_get(const rp_batch *b, rp_batch_info *out)
{
    if (!b || !out) return RP_ERR_INVALID_ARG;
    out->num_items = b->n;
    out->total_sources = b->S_total;
    out->num_groups = (int)b->groups.size();
    unsigned long long rays = 0;
    for (auto &J : b->h_jobs) rays += J.num_rays;
    out->total_rays = rays;
    out->max_group_reflections = b->zmax.hit_cap;
    return RP_OK;
}

int rp_batch_autotune(rp_batch *b, uint64_t seed, const char *cache_path, rp_batch_tuning *best, double *best_ms)
{
    if (!b) return RP_ERR_INVALID_ARG;
    if (cudaSetDevice(b->ctx->device) != cudaSuccess) return RP_ERR_CUDA;
    const std::string key = tuning_key(b);
    rp_batch_tuning t;
    double ms = 0.0;
    int rc;
    if (cache_lookup(cache_path, key, t, ms) && tuning_valid(b, t)) {
        if ((rc = rp_batch_set_tuning(b, &t))) return rc;
        if (best) *best = t;
        if (best_ms) *best_ms = ms;
        return RP_OK;
    }
    cudaStream_t st = batch_stream(b);
    cudaEvent_t e0, e1;
    CKB(cudaEventCreate(&e0));
    CKB(cudaEventCreate(&e1));
    auto time_it = [&](const rp_batch_tuning &x, double &out_ms) -> int {
        int r = rp_batch_set_tuning(b, &x);
        if (r) return r;
        if ((r = run_once(b, seed, 0))) return r;  // warm (and checks the shape runs)
        cudaEventRecord(e0, st);
        if ((r = run_once(b, seed, 0))) return r;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return RP_ERR_CUDA;
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        out_ms = f;
        return RP_OK;
    };
    rp_batch_tuning cur = b->tuning;
    double cur_ms = 0.0;
    if ((rc = time_it(cur, cur_ms))) goto done;
    {
        // coordinate descent over the launch-shape knobs
        const int pocc = paths_occupancy(b->common.flags), socc = shadow_occupancy(b->common.flags);
        const std::vector<int> steps = {4, 8, 16};
        const std::vector<int> chunks = {64, 256, 1024};
        const std::vector<int> pb = {pocc, std::max(1, pocc / 2)};
        const std::vector<int> sb = {socc, std::max(1, socc / 2)};
        const std::vector<int> modes = {1, 2};
        for (int knob = 0; knob < 5; ++knob) {
            const std::vector<int> &cand = knob == 0 ? modes : knob == 1 ? steps : knob == 2 ? chunks
                                         : knob == 3 ? pb : sb;
            for (int v : cand) {
                rp_batch_tuning x = cur;
                int &field = knob == 0 ? x.shadow_mode : knob == 1 ? x.shadow_steps : knob == 2 ? x.chunk_rays
                                       : knob == 3 ? x.paths_blocks_per_sm : x.shadow_blocks_per_sm;
                if (field == v) continue;
                field = v;
                if (!tuning_valid(b, x)) continue;
                double m = 0.0;
                if ((rc = time_it(x, m))) goto done;
                if (m < cur_ms) {
                    cur = x;
                    cur_ms = m;
                }
            }
        }
    }
    rc = rp_batch_set_tuning(b, &cur);
    if (!rc) cache_store(cache_path, key, cur, cur_ms);
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"
