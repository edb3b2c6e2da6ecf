// api.cu -- the C ABI (include/rpr.h): contexts, scenes, workspace, the trace step
// orchestration, estimation, host-buffer updates and kernel timing.
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

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return RP_OK;
    if (e == cudaErrorMemoryAllocation) return RP_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInvalidDevice || e == cudaErrorNoKernelImageForDevice ||
        e == cudaErrorInsufficientDriver)
        return RP_ERR_NO_DEVICE;
    return RP_ERR_CUDA;
}

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

int ensure(rp_ctx *c, Buf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return RP_OK;
    CK(cudaStreamSynchronize(c->stream));
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    CK(cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
    c->ws_gen++;
    return RP_OK;
}

void free_buf(Buf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

void prof_collect(rp_ctx *c)
{
    if (c->pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto &t = c->totals[p.name];
            t.first += 1;
            t.second += ms;
        }
        c->free_events.push_back(p.a);
        c->free_events.push_back(p.b);
    }
    c->pending.clear();
}

// Store passes of the planned refill (one job, FP64 paths, no hashes or visit counts):
// reflection slots past the budget N M for the paths of candidates the waves do not
// take (N M / 16 + 2^20), and one SpecRays slot per speculative candidate
// (max(4 N, 8192), at most N M).
bool store_capable(const rp_trace_params *p)
{
    const unsigned long long budget = p->num_rays * (unsigned long long)std::max(p->max_order, 0);
    return p->budget_refill && budget > 0 && budget <= PLAN_MAX_RAYS &&
           !(p->flags & (RP_FLAG_FP32_PATHS | RP_FLAG_COUNT_VISITS | RP_FLAG_RAY_HASH));
}

StepSizes trace_sizes(const rp_scene *sc, const rp_trace_params *p, int S)
{
    const unsigned long long rays = p->num_rays;
    const int K = (p->sh_order + 1) * (p->sh_order + 1);
    StepSizes z = step_sizes(&rays, &S, 1, p->max_order, sc->B, K, p->num_bins, REC_BUDGET);
    if (store_capable(p)) z.hit_cap += rays * (unsigned long long)p->max_order / 16 + (1ull << 20);
    return z;
}

unsigned long long spec_slots(const rp_trace_params *p)
{
    const unsigned long long budget = p->num_rays * (unsigned long long)std::max(p->max_order, 0);
    return std::min(budget, std::max(4ull * p->num_rays, 8192ull));
}

// The refill planner's buffers: each candidate's segments (plan_seg) and the store
// passes' speculative rays (spec; none when early reflections are kept or test limits
// shrink the capacities).  w = NULL: reserve only.
int bind_planner(rp_ctx *c, const rp_scene *sc, const rp_trace_params *p, bool early, TraceWork *w)
{
    if (w) {
        w->plan = 0;
        w->plan_seg = nullptr;
        w->spec = SpecRays{};
    }
    const unsigned long long budget = p->num_rays * (unsigned long long)std::max(p->max_order, 0);
    if (!p->budget_refill || budget == 0 || budget > PLAN_MAX_RAYS) return RP_OK;
    int rc;
    if ((rc = ensure(c, c->plan_seg, budget * sizeof(uint32_t)))) return rc;
    if (w) w->plan_seg = (uint32_t *)c->plan_seg.p;
    if (!store_capable(p) || early || c->dbg.hit_cap != 0 || c->dbg.record_cap != 0 || c->dbg.spec_slots < 0)
        return RP_OK;
    const unsigned long long cap =
        c->dbg.spec_slots > 0 ? std::min<unsigned long long>(c->dbg.spec_slots, spec_slots(p)) : spec_slots(p);
    if ((rc = ensure(c, c->spec, spec_bytes(cap, sc->B)))) return rc;
    if (!w) return RP_OK;
    const size_t B = (size_t)sc->B;
    char *q = (char *)c->spec.p;
    SpecRays &r = w->spec;
    r.saved = (rp_trace_stats *)q;
    q += sizeof(rp_trace_stats);
    r.late = (double *)q;
    q += cap * B * sizeof(double);
    r.L = (double *)q;
    q += cap * sizeof(double);
    r.t1 = (double *)q;
    q += cap * sizeof(double);
    r.w = (float *)q;
    q += cap * B * sizeof(float);
    r.absb = (float *)q;
    q += cap * B * sizeof(float);
    r.esc = (uint32_t *)q;
    q += cap * sizeof(uint32_t);
    r.sph = (uint32_t *)q;
    q += cap * sizeof(uint32_t);
    r.rerun = (uint32_t *)q;
    r.cap = cap;
    return RP_OK;
}

// make the context workspace hold a group of these sizes with `njobs` jobs
int reserve(rp_ctx *c, const StepSizes &z, int B, int njobs, int total_sources, int nchunks)
{
    int r;
    if ((r = ensure(c, c->hit_p, z.hit_cap * sizeof(float4)))) return r;
    if ((r = ensure(c, c->hit_plo, z.hit_cap * sizeof(float4)))) return r;
    if ((r = ensure(c, c->hit_n, z.hit_cap * sizeof(float4)))) return r;
    if ((r = ensure(c, c->hit_ws, z.hit_cap * B * sizeof(float)))) return r;
    if ((r = ensure(c, c->hit_rid, z.hit_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->hord_cell, z.hit_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->shit_p, z.hit_cap * sizeof(float4)))) return r;
    if ((r = ensure(c, c->hord_perm, z.hit_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->shit_n, z.hit_cap * sizeof(float4)))) return r;
    if ((r = ensure(c, c->shit_ws, z.hit_cap * B * sizeof(float)))) return r;
    if ((r = ensure(c, c->shit_rid, z.hit_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->hord_cnt, (size_t)(hit_order_cells(njobs) + 1) * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->rec_key, z.rec_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->rec_rid, z.rec_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->rec_e, z.rec_cap * B * sizeof(float)))) return r;
    if ((r = ensure(c, c->perm, z.rec_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->rerun, z.rerun_cap * sizeof(unsigned long long)))) return r;
    if ((r = ensure(c, c->cnt, (z.keys + 1) * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->cur, z.keys * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->segkey, z.seg_cap * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->seg_s, z.seg_cells * sizeof(float)))) return r;
    if ((r = ensure(c, c->seg_e, z.seg_cells * sizeof(float)))) return r;
    if ((r = ensure(c, c->off, (z.keys + 1) * sizeof(uint32_t)))) return r;
    if ((r = ensure(c, c->scan_part,
                    scan_parts(std::max<unsigned long long>(z.keys, hit_order_cells(njobs))) * sizeof(uint32_t))))
        return r;
    if ((r = ensure(c, c->Hs, z.cells * sizeof(float)))) return r;
    if ((r = ensure(c, c->He, z.cells * sizeof(float)))) return r;
    if ((r = ensure(c, c->src, (size_t)(total_sources + njobs) * sizeof(float4)))) return r;
    if ((r = ensure(c, c->src_job, (size_t)std::max(total_sources, 1) * sizeof(int)))) return r;
    if ((r = ensure(c, c->src_node, (1 + SRC_HINT_STRIDE) * (size_t)std::max(total_sources, 1) * sizeof(int))))
        return r;
    if ((r = ensure(c, c->jobs, (size_t)njobs * sizeof(SceneJob)))) return r;
    if ((r = ensure(c, c->js, (size_t)njobs * sizeof(JobState)))) return r;
    if ((r = ensure(c, c->chunks, (size_t)std::max(nchunks, 1) * sizeof(RayChunk)))) return r;
    if ((r = ensure(c, c->ctr, sizeof(TraceCounters)))) return r;
    if ((r = ensure(c, c->stats, sizeof(rp_trace_stats)))) return r;
    return RP_OK;
}

// bind the context workspace into a TraceWork for a group of these sizes
void bind_workspace(rp_ctx *c, const StepSizes &z, TraceWork &w)
{
    w.ctr = (TraceCounters *)c->ctr.p;
    w.hits = {(float4 *)c->hit_p.p, (float4 *)c->hit_plo.p, (float4 *)c->hit_n.p, (float *)c->hit_ws.p,
              (uint32_t *)c->hit_rid.p, z.hit_cap};
    w.rec = {(uint32_t *)c->rec_key.p, (uint32_t *)c->rec_rid.p, (float *)c->rec_e.p, z.rec_cap};
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
    w.seg_cap = z.seg_cap;
    w.items_per_chunk = z.items_per_chunk;
    w.rerun = (unsigned long long *)c->rerun.p;
    w.rerun_cap = z.rerun_cap;
    w.num_sms = c->num_sms;
    w.jobs = (const SceneJob *)c->jobs.p;
    w.js = (JobState *)c->js.p;
    w.chunks = (const RayChunk *)c->chunks.p;
    w.src_job = (const int *)c->src_job.p;
    w.src_node = (int *)c->src_node.p;
    // the hints after the start nodes (the buffer holds at least as many sources as this step)
    w.src_hint = (int *)c->src_node.p + (c->src_node.bytes / sizeof(int)) / (1 + SRC_HINT_STRIDE);
    w.region_frac = c->region_frac;
    w.escalate = c->escalate;
    w.pos = (const float4 *)c->src.p;
    w.shits = {(float4 *)c->shit_p.p, nullptr, (float4 *)c->shit_n.p, (float *)c->shit_ws.p,
               (uint32_t *)c->shit_rid.p, z.hit_cap};
    w.horder = {(uint32_t *)c->hord_cell.p, (uint32_t *)c->hord_perm.p, (uint32_t *)c->hord_cnt.p, hit_order_bits(1),
                (int)hit_order_cells(1)};
}

void fill_consts(const rp_scene *sc, const rp_trace_params *p, int S, TraceWork &w)
{
    w.k.S = S;
    w.k.B = sc->B;
    w.k.K = (p->sh_order + 1) * (p->sh_order + 1);
    w.k.T = p->num_bins;
    w.k.M = p->max_order;
    w.k.min_order = p->min_order;
    w.k.sh_order = p->sh_order;
    w.k.rate = p->ir_rate_hz;
    w.k.c = p->speed_of_sound;
    w.k.rs = p->source_radius;
    w.k.flags = p->flags;
}

SceneView scene_view(const rp_scene *sc)
{
    return make_view(sc);
}

void prof_hook(void *ctx, const char *name, int begin)
{
    rp_ctx *c = (rp_ctx *)ctx;
    if (!c->prof) return;
    cudaEvent_t e = get_event(c);
    cudaEventRecord(e, c->stream);
    if (begin) {
        c->open_events.push_back({name, e, nullptr});
    } else if (!c->open_events.empty()) {
        ProfPair pp = c->open_events.back();
        c->open_events.pop_back();
        pp.b = e;
        c->pending.push_back(pp);
    }
}

int check_params(const rp_scene *sc, const rp_trace_params *p, int S)
{
    if (!sc || !p) return RP_ERR_INVALID_ARG;
    if (S < 0 || S > RP_MAX_SOURCES) return RP_ERR_INVALID_ARG;
    if (p->max_order < 0 || p->sh_order < 0 || p->sh_order > RP_MAX_SH_ORDER) return RP_ERR_INVALID_ARG;
    if (p->num_bins < 1 || p->min_order < 0) return RP_ERR_INVALID_ARG;
    if ((p->flags & RP_FLAG_SHADOW_PACKETS) && (p->flags & RP_FLAG_SHADOW_LANES)) return RP_ERR_INVALID_ARG;
    if ((unsigned long long)S * (unsigned long long)p->num_bins >= (1ull << 31)) return RP_ERR_INVALID_ARG;
    // ray ids are 32-bit: first_ray + num_rays <= 2^32, written so that it cannot wrap
    if (p->num_rays > 0xffffffffull || p->first_ray > 0x100000000ull - p->num_rays) return RP_ERR_INVALID_ARG;
    if (p->num_rays * (unsigned long long)std::max(p->max_order, 1) >= (1ull << 40)) return RP_ERR_INVALID_ARG;
    // the refill waves continue the ids after the first wave: at most N M rays in all
    if (p->budget_refill && p->num_rays * (unsigned long long)std::max(p->max_order, 0) > 0x100000000ull - p->first_ray)
        return RP_ERR_INVALID_ARG;
    if (!(p->ir_rate_hz > 0.f) || !(p->speed_of_sound > 0.f) || !(p->source_radius > 0.f))
        return RP_ERR_INVALID_ARG;
    if (!std::isfinite(p->ir_rate_hz) || !std::isfinite(p->speed_of_sound) || !std::isfinite(p->source_radius))
        return RP_ERR_NAN_INPUT;
    return RP_OK;
}

__global__ void k_pack_positions(const float *lis, const float *src, int S, float4 *out, int *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > S) return;
    const float *p = i < S ? src + 3 * i : lis;
    const float x = p[0], y = p[1], z = p[2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) raise_error(status, RP_ERR_NAN_INPUT);
    out[i] = make_float4(x, y, z, 0.f);
}


}  // namespace

extern "C" {

const char *rp_status_string(int s)
{
    switch (s) {
    case RP_OK: return "ok";
    case RP_ERR_INVALID_ARG: return "invalid argument";
    case RP_ERR_CUDA: return "CUDA error";
    case RP_ERR_OOM: return "out of device memory";
    case RP_ERR_CAPACITY: return "internal buffer capacity exceeded";
    case RP_ERR_STACK_OVERFLOW: return "BVH traversal stack overflow";
    case RP_ERR_TIMEOUT: return "traversal iteration cap reached";
    case RP_ERR_NAN_INPUT: return "non-finite input";
    case RP_ERR_EMPTY_SCENE: return "scene has no triangles";
    case RP_ERR_NO_DEVICE: return "no usable CUDA device";
    case RP_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of rp_trace_noalloc";
    case RP_ERR_BOUNDS: return "index out of range (bounds-checked build)";
    default: return "unknown status";
    }
}

int rp_create(rp_ctx **out, int device, void *cuda_stream)
{
    if (!out) return RP_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0 || device < 0 || device >= n) return RP_ERR_NO_DEVICE;
    CK(cudaSetDevice(device));
    rp_ctx *c = new (std::nothrow) rp_ctx();
    if (!c) return RP_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMalloc(&c->d_status, sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return cuda_status(e);
    }
    cudaMemset(c->d_status, 0, sizeof(int));
    c->paths_blocks = c->num_sms * paths_occupancy(0);
    c->shadow_blocks = c->num_sms * shadow_occupancy(0);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return cuda_status(e);
    }
    *out = c;
    return RP_OK;
}

int rp_destroy(rp_ctx *c)
{
    if (!c) return RP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (Buf *b : {&c->hit_p, &c->hit_plo, &c->hit_n, &c->hit_ws, &c->hit_rid, &c->shit_p, &c->hord_perm,
                   &c->shit_n, &c->shit_ws, &c->shit_rid, &c->hord_cell, &c->hord_cnt, &c->rec_key, &c->rec_rid,
                   &c->rec_e, &c->perm, &c->rerun,
                   &c->cnt, &c->off, &c->cur, &c->scan_part, &c->Hs, &c->He, &c->src, &c->ctr, &c->stats, &c->H,
                   &c->direct,
                   &c->params, &c->state, &c->jobs, &c->js, &c->chunks, &c->src_job, &c->src_node, &c->plan_seg, &c->spec, &c->segkey, &c->seg_s, &c->seg_e, &c->rv_raw,
                   &c->rv_bands, &c->rv_comb, &c->rv_ap, &c->rv_phi})
        free_buf(*b);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->free_events) cudaEventDestroy(e);
    cudaFree(c->d_status);
    delete c;
    return RP_OK;
}

int rp_set_debug_limits(rp_ctx *c, const rp_debug_limits *lim)
{
    if (!c) return RP_ERR_INVALID_ARG;
    if (!lim) {
        c->dbg = rp_debug_limits{0, 0, 0ull, 0ull};
        return RP_OK;
    }
    if (lim->iter_cap < 0 || lim->spec_slots < -1) return RP_ERR_INVALID_ARG;
    c->dbg = *lim;
    return RP_OK;
}

int rp_set_stream(rp_ctx *c, void *cuda_stream)
{
    if (!c) return RP_ERR_INVALID_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return RP_OK;
}

int rp_sync_status(rp_ctx *c)
{
    if (!c) return RP_ERR_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    int h = 0;
    CK(cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) CK(cudaMemset(c->d_status, 0, sizeof(int)));
    return h;
}

int rp_scene_create(rp_ctx *c, const rp_mesh_desc *m, rp_scene **out)
{
    if (!c || !m || !out) return RP_ERR_INVALID_ARG;
    *out = nullptr;
    if (m->num_tris == 0) return RP_ERR_EMPTY_SCENE;
    if (m->num_tris < 0 || m->num_verts <= 0 || m->num_materials <= 0 || m->num_bands < 1 ||
        m->num_bands > RP_MAX_BANDS || !m->verts || !m->tris || !m->tri_material || !m->absorption ||
        !m->scattering || (m->memory != RP_MEM_HOST && m->memory != RP_MEM_DEVICE))
        return RP_ERR_INVALID_ARG;
    if (!std::isfinite(m->ray_epsilon) || m->ray_epsilon < 0.f) return RP_ERR_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    const int nv = m->num_verts, nt = m->num_tris, nm = m->num_materials, B = m->num_bands;
    const float *dv = m->verts, *da = m->absorption, *ds = m->scattering;
    const int32_t *dt = m->tris, *dm = m->tri_material;
    void *tmp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int rc = RP_OK;
    rp_scene *sc = new (std::nothrow) rp_scene();
    if (!sc) return RP_ERR_OOM;
    sc->ctx = c;
    sc->num_tris = nt;
    sc->num_nodes = nt - 1;
    sc->num_mats = nm;
    sc->B = B;
    sc->num_verts = nv;
    sc->ray_eps = m->ray_epsilon;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BvhBuildArgs a;
    BvhOut o;
    cudaError_t err;
    if (m->memory == RP_MEM_HOST) {
        const size_t sz[5] = {sizeof(float) * 3 * nv, sizeof(int32_t) * 3 * nt, sizeof(int32_t) * nt,
                              sizeof(float) * nm * B, sizeof(float) * nm * B};
        const void *src[5] = {m->verts, m->tris, m->tri_material, m->absorption, m->scattering};
        for (int i = 0; i < 5; ++i) {
            if ((err = cudaMalloc(&tmp[i], sz[i])) != cudaSuccess) { rc = cuda_status(err); goto fail; }
            if ((err = cudaMemcpyAsync(tmp[i], src[i], sz[i], cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) {
                rc = cuda_status(err);
                goto fail;
            }
        }
        dv = (const float *)tmp[0];
        dt = (const int32_t *)tmp[1];
        dm = (const int32_t *)tmp[2];
        da = (const float *)tmp[3];
        ds = (const float *)tmp[4];
    }
    if ((err = cudaMalloc(&sc->nodes, sizeof(float4) * 4 * (size_t)std::max(nt - 1, 1))) != cudaSuccess ||
        (err = cudaMalloc(&sc->tris, sizeof(float4) * 3 * (size_t)nt)) != cudaSuccess ||
        (err = cudaMalloc(&sc->alpha, sizeof(float) * nm * B)) != cudaSuccess ||
        (err = cudaMalloc(&sc->scat, sizeof(float) * nm * B)) != cudaSuccess ||
        (err = cudaMalloc(&sc->wdiff, sizeof(float) * nm * B)) != cudaSuccess ||
        (err = cudaMalloc(&sc->wspec, sizeof(float) * nm * B)) != cudaSuccess ||
        (err = cudaMalloc(&sc->thr, sizeof(uint32_t) * nm)) != cudaSuccess ||
        (err = cudaMalloc(&sc->vidx, sizeof(int32_t) * 3 * (size_t)nt)) != cudaSuccess ||
        (err = cudaMalloc(&sc->pleaf, sizeof(int) * (size_t)nt)) != cudaSuccess ||
        (err = cudaMalloc(&sc->pint, sizeof(int) * (size_t)std::max(nt - 1, 1))) != cudaSuccess ||
        (err = cudaMalloc(&sc->anc, sizeof(int) * (size_t)nt)) != cudaSuccess ||
        (err = cudaMalloc(&sc->up, sizeof(int) * (size_t)std::max(nt - 1, 1))) != cudaSuccess ||
        (err = cudaMemcpyAsync(sc->vidx, dt, sizeof(int32_t) * 3 * (size_t)nt, cudaMemcpyDeviceToDevice,
                               c->stream)) != cudaSuccess) {
        rc = cuda_status(err);
        goto fail;
    }
    a = {dv, dt, dm, da, ds, nv, nt, nm, B, m->ray_epsilon};
    o.nodes = sc->nodes;
    o.tris = sc->tris;
    o.alpha = sc->alpha;
    o.scat = sc->scat;
    o.wdiff = sc->wdiff;
    o.wspec = sc->wspec;
    o.thr = sc->thr;
    o.pleaf = sc->pleaf;
    o.pint = sc->pint;
    o.anc = sc->anc;
    o.up = sc->up;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    cudaEventRecord(e0, c->stream);
    err = build_bvh(a, o, c->d_status, c->stream);
    cudaEventRecord(e1, c->stream);
    if (err != cudaSuccess) {
        rc = cuda_status(err);
        goto fail;
    }
    if ((rc = rp_sync_status(c)) != RP_OK) goto fail;
    cudaEventElapsedTime(&sc->build_ms, e0, e1);
    sc->tmin = o.tmin;
    sc->tmin_d = o.tmin_d;
    sc->max_depth = o.max_depth;
    for (int k = 0; k < 3; ++k) {
        sc->lo[k] = o.lo[k];
        sc->hi[k] = o.hi[k];
    }
    for (void *p : tmp) cudaFree(p);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = sc;
    return RP_OK;
fail:
    cudaStreamSynchronize(c->stream);
    for (void *p : tmp) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    rp_scene_destroy(sc);
    return rc;
}

int rp_scene_destroy(rp_scene *sc)
{
    if (!sc) return RP_ERR_INVALID_ARG;
    cudaSetDevice(sc->ctx->device);
    cudaStreamSynchronize(sc->ctx->stream);
    cudaFree(sc->nodes);
    cudaFree(sc->tris);
    cudaFree(sc->alpha);
    cudaFree(sc->scat);
    cudaFree(sc->wdiff);
    cudaFree(sc->wspec);
    cudaFree(sc->thr);
    cudaFree(sc->vidx);
    cudaFree(sc->pleaf);
    cudaFree(sc->pint);
    cudaFree(sc->anc);
    cudaFree(sc->up);
    delete sc;
    return RP_OK;
}

int rp_scene_info_get(const rp_scene *sc, rp_scene_info *out)
{
    if (!sc || !out) return RP_ERR_INVALID_ARG;
    out->num_tris = sc->num_tris;
    out->num_nodes = sc->num_nodes;
    out->max_depth = sc->max_depth;
    out->num_bands = sc->B;
    for (int k = 0; k < 3; ++k) {
        out->bounds_lo[k] = sc->lo[k];
        out->bounds_hi[k] = sc->hi[k];
    }
    out->ray_epsilon = sc->tmin;
    out->build_ms = sc->build_ms;
    out->refit_ms = sc->refit_ms;
    return RP_OK;
}

int rp_trace_reserve(rp_scene *sc, const rp_trace_params *p, int32_t S)
{
    int rc = check_params(sc, p, S);
    if (rc) return rc;
    CK(cudaSetDevice(sc->ctx->device));
    if ((rc = reserve(sc->ctx, trace_sizes(sc, p, S), sc->B, 1, S, 1))) return rc;
    return bind_planner(sc->ctx, sc, p, false, nullptr);
}

}  // extern "C"

// The trace step of rp_trace, optionally keeping early reflections (rp_trace_er);
// *work_out receives the step's bindings (device counters, positions, job state).
int rp::trace_enqueue(rp_scene *sc, const rp_trace_params *p, const float *listener, const float *sources, int32_t S,
                      float *H, rp_direct *direct, rp_trace_stats *stats, uint64_t *ray_hash, const EarlyHits *early,
                      TraceWork *work_out)
{
    int rc = check_params(sc, p, S);
    if (rc) return rc;
    if (!listener || (S > 0 && !sources) || (!H && S > 0)) return RP_ERR_INVALID_ARG;
    rp_ctx *c = sc->ctx;
    CK(cudaSetDevice(c->device));
    const StepSizes z = trace_sizes(sc, p, S);
    if ((rc = reserve(c, z, sc->B, 1, S, 1))) return rc;
    cudaStream_t st = c->stream;

    TraceWork w;
    bind_workspace(c, z, w);
    fill_consts(sc, p, S, w);
    // positions: sources then the listener, packed as float4 on the device
    float4 *dsrc = (float4 *)c->src.p;
    if (p->flags & RP_FLAG_DEVICE_POSITIONS) {
        ProfScope ps(c, "pack_positions");
        k_pack_positions<<<(S + 1 + 127) / 128, 128, 0, st>>>(listener, sources, S, dsrc, c->d_status);
    } else {
        std::vector<float4> hp(S + 1);
        for (int i = 0; i <= S; ++i) {
            const float *q = i < S ? sources + 3 * i : listener;
            if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2])) return RP_ERR_NAN_INPUT;
            hp[i] = make_float4(q[0], q[1], q[2], 0.f);
        }
        // from pageable memory the copy is staged before the call returns
        CK(cudaMemcpyAsync(dsrc, hp.data(), sizeof(float4) * (S + 1), cudaMemcpyHostToDevice, st));
    }
    SceneJob job;
    job.sc = scene_view(sc);
    job.first_ray = p->first_ray;
    job.num_rays = p->num_rays;
    job.hit_off = 0;
    job.hit_cap = z.hit_cap;
    // test limits (rp_set_debug_limits): a smaller iteration cap or capacity
    if (c->dbg.iter_cap > 0) job.sc.iter_cap = c->dbg.iter_cap;
    if (c->dbg.hit_cap > 0) job.hit_cap = std::min<unsigned long long>(job.hit_cap, c->dbg.hit_cap);
    if (c->dbg.record_cap > 0) w.rec.cap = std::min<unsigned long long>(w.rec.cap, c->dbg.record_cap);
    job.scene_id = p->scene_id;
    job.S = S;
    job.src_off = 0;
    job.lis = S;
    CK(cudaMemcpyAsync(c->jobs.p, &job, sizeof(SceneJob), cudaMemcpyHostToDevice, st));
    w.job0 = job;
    w.njobs = 1;
    w.wave_mode = 1;
    w.nchunks = 0;
    w.chunk_rays = 1;
    w.src_base = 0;
    w.seed = nullptr;
    w.seed_val = p->seed;
    w.ray_hash = (p->flags & RP_FLAG_RAY_HASH) ? ray_hash : nullptr;
    w.H = H;
    w.direct = direct;
    w.shadow_steps = c->shadow_steps;
    w.shadow_packets = shadow_packets_for(p->flags);
    w.plan = 0;
    w.plan_seg = nullptr;
    if ((rc = bind_planner(c, sc, p, early != nullptr, &w))) return rc;

    StepLaunch L;
    L.w = w;
    L.n_rec_chunks = z.n_chunks;
    L.refill = p->budget_refill;
    L.reset_stats = 1;
    L.paths_blocks = c->paths_blocks;
    L.shadow_blocks = c->shadow_blocks;
    L.exact_blocks = c->num_sms * 2;
    L.flat_blocks = c->num_sms * 8;
    L.acc_blocks = (int)std::max(1ll, std::min<long long>(((long long)z.keys + 7) / 8, (long long)c->num_sms * 8));
    if (early) {
        L.w.er = *early;
        w.er = *early;
    }
    CK(enqueue_step(L, st, prof_hook, c));
    if (stats) CK(cudaMemcpyAsync(stats, w.stats, sizeof(rp_trace_stats), cudaMemcpyDeviceToDevice, st));
    if (work_out) *work_out = w;
    return RP_OK;
}

extern "C" {

int rp_trace(rp_scene *sc, const rp_trace_params *p, const float *listener, const float *sources, int32_t S,
             float *H, rp_direct *direct, rp_trace_stats *stats, uint64_t *ray_hash)
{
    return trace_enqueue(sc, p, listener, sources, S, H, direct, stats, ray_hash, nullptr, nullptr);
}

int rp_estimate(rp_ctx *c, const float *H, const rp_direct *direct, int32_t S, int32_t B, int32_t K, int32_t T,
                const rp_estimate_params *ep, rp_reverb_params *out, double *state)
{
    if (!c || !ep || (S > 0 && (!H || !out))) return RP_ERR_INVALID_ARG;
    if (S < 0 || B < 1 || B > RP_MAX_BANDS || K < 1 || K > RP_MAX_SH || T < 1) return RP_ERR_INVALID_ARG;
    const int n = (int)std::lround(std::sqrt((double)K));
    if (n * n != K) return RP_ERR_INVALID_ARG;
    if (!(ep->ir_rate_hz > 0.0) || ep->tau < 0.0 || ep->dt_update < 0.0) return RP_ERR_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    EstimateWork w{H, direct, S, B, K, T, ep->ir_rate_hz, ep->dt_update, ep->tau, out, state};
    {
        ProfScope ps(c, "estimate");
        launch_estimate(w, c->stream);
    }
    CK(cudaGetLastError());
    return RP_OK;
}

int rp_update(rp_scene *sc, const rp_trace_params *p, const rp_estimate_params *ep, const float *listener,
              const float *sources, int32_t S, float *H_host, rp_reverb_params *params_host, rp_direct *direct_host,
              rp_trace_stats *stats_host, double *state_host)
{
    int rc = check_params(sc, p, S);
    if (rc) return rc;
    if (!ep || (p->flags & RP_FLAG_DEVICE_POSITIONS)) return RP_ERR_INVALID_ARG;
    rp_ctx *c = sc->ctx;
    CK(cudaSetDevice(c->device));
    const int K = (p->sh_order + 1) * (p->sh_order + 1);
    const size_t cells = (size_t)S * sc->B * K * p->num_bins;
    if ((rc = ensure(c, c->H, cells * sizeof(float)))) return rc;
    if ((rc = ensure(c, c->direct, (size_t)std::max(S, 1) * sizeof(rp_direct)))) return rc;
    if ((rc = ensure(c, c->params, (size_t)std::max(S, 1) * sc->B * sizeof(rp_reverb_params)))) return rc;
    if ((rc = ensure(c, c->state, (size_t)std::max(S, 1) * sc->B * sizeof(double)))) return rc;
    cudaStream_t st = c->stream;
    double *dstate = nullptr;
    if (state_host) {
        dstate = (double *)c->state.p;
        CK(cudaMemcpyAsync(dstate, state_host, sizeof(double) * S * sc->B, cudaMemcpyHostToDevice, st));
    }
    rp_trace_params q = *p;
    q.flags &= ~RP_FLAG_RAY_HASH;
    if ((rc = rp_trace(sc, &q, listener, sources, S, (float *)c->H.p, (rp_direct *)c->direct.p, nullptr, nullptr)))
        return rc;
    if ((rc = rp_estimate(c, (float *)c->H.p, (rp_direct *)c->direct.p, S, sc->B, K, p->num_bins, ep,
                          (rp_reverb_params *)c->params.p, dstate)))
        return rc;
    if (H_host) CK(cudaMemcpyAsync(H_host, c->H.p, cells * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (params_host)
        CK(cudaMemcpyAsync(params_host, c->params.p, sizeof(rp_reverb_params) * S * sc->B, cudaMemcpyDeviceToHost,
                           st));
    if (direct_host) CK(cudaMemcpyAsync(direct_host, c->direct.p, sizeof(rp_direct) * S, cudaMemcpyDeviceToHost, st));
    if (stats_host)
        CK(cudaMemcpyAsync(stats_host, c->stats.p, sizeof(rp_trace_stats), cudaMemcpyDeviceToHost, st));
    if (state_host) CK(cudaMemcpyAsync(state_host, dstate, sizeof(double) * S * sc->B, cudaMemcpyDeviceToHost, st));
    return rp_sync_status(c);
}

int rp_profile_enable(rp_ctx *c, int enable)
{
    if (!c) return RP_ERR_INVALID_ARG;
    c->prof = enable != 0;
    return RP_OK;
}

int rp_profile_reset(rp_ctx *c)
{
    if (!c) return RP_ERR_INVALID_ARG;
    prof_collect(c);
    c->totals.clear();
    return RP_OK;
}

int rp_profile_read(rp_ctx *c, rp_kernel_time *out, int32_t max_entries, int32_t *count)
{
    if (!c || !count || (max_entries > 0 && !out)) return RP_ERR_INVALID_ARG;
    prof_collect(c);
    int i = 0;
    for (auto &kv : c->totals) {
        if (i < max_entries) {
            std::memset(out[i].name, 0, sizeof(out[i].name));
            std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.first;
            out[i].total_ms = kv.second.second;
        }
        ++i;
    }
    *count = i;
    return RP_OK;
}

}  // extern "C"
