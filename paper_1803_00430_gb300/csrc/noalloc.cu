// noalloc.cu -- rp_trace_noalloc: the trace step with its scratch memory in a fixed,
// statically allocated device array instead of library-allocated workspace.
//
// rp_trace allocates (and grows) device workspace with cudaMalloc the first time a
// problem size is seen.  Some callers cannot allow that: a real-time audio or game
// thread that must never block on the driver's allocator mid-frame, or a host
// application that hands out all device memory from a pool of its own and forbids
// libraries to allocate behind its back.
// rp_trace_noalloc runs the same kernels on the same inputs and writes the same
// outputs, but takes every temporary buffer (counters, stored reflections,
// contribution records, the counting sort, the compensated sums) from one
// file-scope __device__ array of RP_NOALLOC_SCRATCH_BYTES.  It calls no cudaMalloc,
// cudaFree or allocating routine, on the device or the host.
//
// Consequences of a shared static array:
//   - every GPU that loads the library holds RP_NOALLOC_SCRATCH_BYTES until exit;
//   - all calls on a device share the one array, which keeps the previous call's
//     contents (this file clears what must start at zero); calls that overlap on
//     the GPU (other streams, other host threads) race on it and must be ordered
//     by the caller;
//   - the device address of the array is looked up once per device, with that
//     device current, on the first call there: make that first call before any
//     stream capture begins.
// Host positions are staged with cudaMemcpyAsync from the caller's arrays, and with
// budget refill the host reads each batch of waves' size back (the stream is
// synchronised), as in rp_trace.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "handles.cuh"

using namespace rp;

// the scratch array of the allocation-free entry point (see above)
static __device__ __align__(256) unsigned char g_noalloc_scratch[RP_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
// cells of the reflection order (2^18: 1 MiB of counts, so that the scratch holds
// useful problem sizes)
constexpr int NOALLOC_CELLS_LOG2 = 18;
std::mutex g_mu;
void *g_scratch_ptr[MAX_DEVICES] = {};

// device address of g_noalloc_scratch on the current device `dev`, looked up once
int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return RP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return RP_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[dev];
    return RP_OK;
}

struct Carve {
    unsigned long long off = 0;
    template <typename T>
    unsigned long long take(unsigned long long count)
    {
        const unsigned long long at = off;
        off += (sizeof(T) * std::max(count, 1ull) + 255ull) & ~255ull;
        return at;
    }
};

__global__ void k_pack_positions_na(const float *lis, const float *src, int S, float4 *out, int *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > S) return;
    const float *p = i < S ? src + 3 * i : lis;
    const float x = p[0], y = p[1], z = p[2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) raise_error(status, RP_ERR_NAN_INPUT);
    out[i] = make_float4(x, y, z, 0.f);
}

#define CKN(x)                                        \
    do {                                              \
        const cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return RP_ERR_CUDA;    \
    } while (0)

}  // namespace

extern "C" int rp_trace_noalloc(rp_scene *sc, const rp_trace_params *p, const float *listener, const float *sources,
                                int32_t S, float *H, rp_direct *direct, rp_trace_stats *stats)
{
    if (!sc || !p || !listener || (S > 0 && (!sources || !H))) return RP_ERR_INVALID_ARG;
    if (S < 0 || S > RP_MAX_SOURCES) return RP_ERR_INVALID_ARG;
    if (p->max_order < 0 || p->sh_order < 0 || p->sh_order > RP_MAX_SH_ORDER || p->num_bins < 1 || p->min_order < 0)
        return RP_ERR_INVALID_ARG;
    // ray ids are 32-bit: first_ray + num_rays <= 2^32, written so that it cannot wrap
    if (p->num_rays > 0xffffffffull || p->first_ray > 0x100000000ull - p->num_rays) return RP_ERR_INVALID_ARG;
    // the refill waves continue the ids after the first wave: at most N M rays in all
    if (p->budget_refill && p->num_rays * (unsigned long long)std::max(p->max_order, 0) > 0x100000000ull - p->first_ray)
        return RP_ERR_INVALID_ARG;
    if ((p->flags & RP_FLAG_SHADOW_PACKETS) && (p->flags & RP_FLAG_SHADOW_LANES)) return RP_ERR_INVALID_ARG;
    if (!(p->ir_rate_hz > 0.f) || !(p->speed_of_sound > 0.f) || !(p->source_radius > 0.f)) return RP_ERR_INVALID_ARG;
    if (!std::isfinite(p->ir_rate_hz) || !std::isfinite(p->speed_of_sound) || !std::isfinite(p->source_radius))
        return RP_ERR_NAN_INPUT;
    rp_ctx *c = sc->ctx;
    const int B = sc->B, K = (p->sh_order + 1) * (p->sh_order + 1), T = p->num_bins, M = p->max_order;
    const unsigned long long rays = p->num_rays;
    // the record budget is what the fixed part of the layout leaves; size it by
    // trying the layout with the whole array first
    StepSizes z = step_sizes(&rays, &S, 1, M, B, K, T, 1ull << 40);
    Carve cv;
    const unsigned long long o_ctr = cv.take<TraceCounters>(1), o_st = cv.take<rp_trace_stats>(1);
    const unsigned long long o_job = cv.take<SceneJob>(1), o_js = cv.take<JobState>(1);
    const unsigned long long o_src = cv.take<float4>(S + 1), o_raw = cv.take<float>(3ull * (S + 1));
    const unsigned long long o_hp = cv.take<float4>(z.hit_cap), o_hl = cv.take<float4>(z.hit_cap),
                             o_hn = cv.take<float4>(z.hit_cap), o_hw = cv.take<float>(z.hit_cap * B),
                             o_hr = cv.take<uint32_t>(z.hit_cap), o_hc = cv.take<uint32_t>(z.hit_cap),
                             o_hk = cv.take<uint32_t>((unsigned long long)hit_order_cells(1, NOALLOC_CELLS_LOG2) + 1);
    const unsigned long long o_sp = cv.take<float4>(z.hit_cap), o_sq = cv.take<uint32_t>(z.hit_cap),
                             o_sn = cv.take<float4>(z.hit_cap), o_sw = cv.take<float>(z.hit_cap * B),
                             o_sr = cv.take<uint32_t>(z.hit_cap);
    const unsigned long long o_cnt = cv.take<uint32_t>(z.keys + 1), o_off = cv.take<uint32_t>(z.keys + 1),
                             o_cur = cv.take<uint32_t>(z.keys);
    const unsigned long long o_part = cv.take<uint32_t>(
        scan_parts(std::max<unsigned long long>(z.keys, hit_order_cells(1, NOALLOC_CELLS_LOG2))));
    const unsigned long long o_hs = cv.take<float>(z.cells), o_he = cv.take<float>(z.cells);
    if (cv.off >= RP_NOALLOC_SCRATCH_BYTES) return RP_ERR_TOO_LARGE;
    // the rest holds contribution records (key, ray, energies, sort index), the FP64
    // re-decision queue (one entry per 8 records) and the segment sums of heavy keys
    // (at most 2 segments of B K sum and error pairs and a key per ACC_SEG records)
    const unsigned long long seg_bytes = 4ull + 8ull * B * K;
    const unsigned long long per_rec =
        4ull + 4ull + 4ull * B + 4ull + 1ull + 16ull + (2ull * seg_bytes + ACC_SEG - 1) / ACC_SEG;
    const unsigned long long fixed = 2ull * seg_bytes + 8ull * 256ull;  // 2 more segments, the arrays' alignment
    if (cv.off + fixed >= RP_NOALLOC_SCRATCH_BYTES) return RP_ERR_TOO_LARGE;
    const unsigned long long rec_room = (RP_NOALLOC_SCRATCH_BYTES - cv.off - fixed) / per_rec;
    if (rec_room < z.sph_cap + (unsigned long long)std::max(S, 1)) return RP_ERR_TOO_LARGE;
    z = step_sizes(&rays, &S, 1, M, B, K, T, rec_room);
    const unsigned long long o_rk = cv.take<uint32_t>(z.rec_cap), o_rr = cv.take<uint32_t>(z.rec_cap),
                             o_re = cv.take<float>(z.rec_cap * B), o_pm = cv.take<uint32_t>(z.rec_cap);
    const unsigned long long o_rq = cv.take<unsigned long long>(z.rerun_cap);
    const unsigned long long o_sk = cv.take<uint32_t>(z.seg_cap), o_ss = cv.take<float>(z.seg_cells),
                             o_se = cv.take<float>(z.seg_cells);
    if (cv.off > RP_NOALLOC_SCRATCH_BYTES) return RP_ERR_TOO_LARGE;

    CKN(cudaSetDevice(c->device));
    unsigned char *base = nullptr;
    int rc = scratch_address(c->device, &base);
    if (rc) return rc;
    cudaStream_t st = c->stream;

    float4 *dsrc = (float4 *)(base + o_src);
    const float *lis = listener, *srcs = sources;
    if (!(p->flags & RP_FLAG_DEVICE_POSITIONS)) {
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(listener[i])) return RP_ERR_NAN_INPUT;
        for (long long i = 0; i < 3ll * S; ++i)
            if (!std::isfinite(sources[i])) return RP_ERR_NAN_INPUT;
        float *raw = (float *)(base + o_raw);
        if (S > 0) CKN(cudaMemcpyAsync(raw, sources, sizeof(float) * 3 * S, cudaMemcpyHostToDevice, st));
        CKN(cudaMemcpyAsync(raw + 3 * S, listener, sizeof(float) * 3, cudaMemcpyHostToDevice, st));
        lis = raw + 3 * S;
        srcs = raw;
    }
    k_pack_positions_na<<<(S + 1 + 127) / 128, 128, 0, st>>>(lis, srcs, S, dsrc, c->d_status);

    TraceWork w;
    SceneJob job;
    job.sc = make_view(sc);
    job.first_ray = p->first_ray;
    job.num_rays = p->num_rays;
    job.hit_off = 0;
    job.hit_cap = z.hit_cap;
    job.scene_id = p->scene_id;
    job.S = S;
    job.src_off = 0;
    job.lis = S;
    // the job table lives in the scratch too; the copy is staged from the stack
    CKN(cudaMemcpyAsync(base + o_job, &job, sizeof(SceneJob), cudaMemcpyHostToDevice, st));
    w.job0 = job;
    w.jobs = (const SceneJob *)(base + o_job);
    w.njobs = 1;
    w.js = (JobState *)(base + o_js);
    w.wave_mode = 1;
    w.plan = 0;
    w.plan_seg = nullptr;  // refill runs as waves here: the scratch holds no plan
    w.chunks = nullptr;
    w.nchunks = 0;
    w.chunk_rays = 1;
    w.src_job = nullptr;
    w.src_base = 0;
    w.k.S = S;
    w.k.B = B;
    w.k.K = K;
    w.k.T = T;
    w.k.M = M;
    w.k.min_order = p->min_order;
    w.k.sh_order = p->sh_order;
    w.k.rate = p->ir_rate_hz;
    w.k.c = p->speed_of_sound;
    w.k.rs = p->source_radius;
    w.k.flags = p->flags & ~RP_FLAG_RAY_HASH;
    w.seed = nullptr;
    w.seed_val = p->seed;
    w.pos = dsrc;
    w.ctr = (TraceCounters *)(base + o_ctr);
    w.hits = {(float4 *)(base + o_hp), (float4 *)(base + o_hl), (float4 *)(base + o_hn), (float *)(base + o_hw),
              (uint32_t *)(base + o_hr), z.hit_cap};
    w.rec = {(uint32_t *)(base + o_rk), (uint32_t *)(base + o_rr), (float *)(base + o_re), z.rec_cap};
    w.stats = (rp_trace_stats *)(base + o_st);
    w.ray_hash = nullptr;
    w.status = c->d_status;
    w.cnt = (uint32_t *)(base + o_cnt);
    w.off = (uint32_t *)(base + o_off);
    w.scan_part = (uint32_t *)(base + o_part);
    w.cur = (uint32_t *)(base + o_cur);
    w.perm = (uint32_t *)(base + o_pm);
    w.Hs = (float *)(base + o_hs);
    w.He = (float *)(base + o_he);
    w.segkey = (uint32_t *)(base + o_sk);
    w.Ss = (float *)(base + o_ss);
    w.Se = (float *)(base + o_se);
    w.seg_cap = z.seg_cap;
    w.H = H;
    w.direct = direct;
    w.items_per_chunk = z.items_per_chunk;
    w.rerun = (unsigned long long *)(base + o_rq);
    w.rerun_cap = z.rerun_cap;
    w.num_sms = c->num_sms;
    w.shadow_steps = c->shadow_steps;
    w.shadow_packets = shadow_packets_for(p->flags);
    w.shits = {(float4 *)(base + o_sp), nullptr, (float4 *)(base + o_sn), (float *)(base + o_sw),
               (uint32_t *)(base + o_sr), z.hit_cap};
    w.horder = {(uint32_t *)(base + o_hc), (uint32_t *)(base + o_sq), (uint32_t *)(base + o_hk),
                hit_order_bits(1, NOALLOC_CELLS_LOG2), (int)hit_order_cells(1, NOALLOC_CELLS_LOG2)};

    StepLaunch L;
    L.w = w;
    L.n_rec_chunks = z.n_chunks;
    L.refill = p->budget_refill;
    L.reset_stats = 1;  // what must start at zero: counters, job state, statistics
    L.paths_blocks = c->paths_blocks;
    L.shadow_blocks = c->shadow_blocks;
    L.exact_blocks = c->num_sms * 2;
    L.flat_blocks = c->num_sms * 8;
    L.acc_blocks = (int)std::max(1ll, std::min<long long>(((long long)z.keys + 7) / 8, (long long)c->num_sms * 8));
    CKN(enqueue_step(L, st, nullptr, nullptr));
    if (stats) CKN(cudaMemcpyAsync(stats, w.stats, sizeof(rp_trace_stats), cudaMemcpyDeviceToDevice, st));
    return RP_OK;
}
