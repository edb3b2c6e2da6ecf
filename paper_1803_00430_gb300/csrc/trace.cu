// trace.cu -- backward path tracing from the listener with diffuse rain
// (Section 5, "Sound Propagation"), direct sound, and the segment-budget waves.
//
// A step runs one or many jobs (scenes with their own sources, listener and ray
// budget) through the same persistent launches; BATCH selects the many-job form.
//
// Kernels of one trace step:
//   k_setup       sets each job's first wave; with budget refill (one job) later
//                 waves spend the unused part of the N*M segment budget on
//                 floor(unused / M) extra primaries (Section 5).
//   k_plan_block, k_refill_plan, k_spec_fold, k_plan_apply
//                 planned refill: store passes of k_paths over candidate rays (each
//                 kept as the real pass would keep it), the waves' sizes from their
//                 segment counts, the speculative candidates inside the waves folded
//                 into the statistics; the rest are dropped.  Without store passes: a
//                 counting pass, then all waves as one.
//   k_paths       persistent: each warp takes 32 primaries at a time from a global
//                 counter; each thread follows its path bounce by bounce: closest
//                 hit, absorption, storage of the reflection for next-event
//                 estimation, then a diffuse (cosine lobe, probability mean(s)) or
//                 specular continuation drawn from Philox(ray, scene, bounce).
//                 Path state in FP64 (default) or FP32 (RP_FLAG_FP32_PATHS).
//                 After a specular choice the next segment also tests the sources
//                 as spheres (the specular image of the source).
//   k_hit_cells, k_hit_scatter, k_hit_gather
//                 order the stored reflections by spatial cell (near-cubic cells,
//                 up to 2^22 per scene) and copy them in that order, so that
//                 neighbouring shadow items start close together.
//   k_shadow_packet / k_shadow
//                 persistent over (reflection, source) pairs in tiles of 32
//                 reflections x sources: the diffuse-rain shadow ray of each stored
//                 reflection to each source, as warp packets (32 rays walk the BVH
//                 together, the child towards the source first) or one ray per
//                 lane; a visible source emits a
//                 contribution record w_b s_b cos / (pi d^2) at arrival time
//                 (L + d) / c.  Rounding-sensitive visibilities go to
//                 k_shadow_exact (FP64).
//   k_direct      visibility and closed-form direct sound per source.
#include "traverse.cuh"

namespace rp {
namespace {

constexpr int PATH_THREADS = 128;
constexpr int SHADOW_THREADS = 128;
// an FP32 arrival time within this many bins of a bin boundary is re-decided in FP64
constexpr float BIN_GUARD = 2e-3f;
constexpr int SHADOW_WINDOW = 256;  // items a warp of k_shadow takes from the chunk at a time

struct BlockAcc {
    double esc[MAXB], absb[MAXB], rem[MAXB], late[MAXB];
    double mfp, mfp_np;
    unsigned long long mfp_cnt, mfp_cnt_np, segs, shadow, contrib, sphere, nodes, tris, walks, steps;
};

__device__ __forceinline__ void acc_init(BlockAcc &a)
{
    const int t = threadIdx.x;
    if (t < MAXB) {
        a.esc[t] = 0.0;
        a.absb[t] = 0.0;
        a.rem[t] = 0.0;
        a.late[t] = 0.0;
    }
    if (t == 0) {
        a.mfp = a.mfp_np = 0.0;
        a.mfp_cnt = a.mfp_cnt_np = a.segs = a.shadow = a.contrib = a.sphere = a.nodes = a.tris = 0ull;
        a.walks = a.steps = 0ull;
    }
}

__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ void acc_flush(BlockAcc &a, rp_trace_stats *st, int B, int which)
{
    __syncthreads();
    const int t = threadIdx.x;
    if (t < B) {
        if (a.esc[t] != 0.0) atomicAdd(&st->escaped[t], a.esc[t]);
        if (a.absb[t] != 0.0) atomicAdd(&st->absorbed[t], a.absb[t]);
        if (a.rem[t] != 0.0) atomicAdd(&st->remaining[t], a.rem[t]);
        if (a.late[t] != 0.0) atomicAdd(&st->late[t], a.late[t]);
    }
    if (t == 0) {
        if (a.mfp != 0.0) atomicAdd(&st->mfp_sum, a.mfp);
        if (a.mfp_np != 0.0) atomicAdd(&st->mfp_sum_np, a.mfp_np);
        if (a.mfp_cnt) atomicAdd((unsigned long long *)&st->mfp_count, a.mfp_cnt);
        if (a.mfp_cnt_np) atomicAdd((unsigned long long *)&st->mfp_count_np, a.mfp_cnt_np);
        if (a.segs) atomicAdd((unsigned long long *)&st->segments, a.segs);
        if (a.shadow) atomicAdd((unsigned long long *)&st->shadow_rays, a.shadow);
        if (a.contrib) atomicAdd((unsigned long long *)&st->contributions, a.contrib);
        if (a.sphere) atomicAdd((unsigned long long *)&st->sphere_hits, a.sphere);
        if (a.nodes) atomicAdd((unsigned long long *)&st->node_visits[which], a.nodes);
        if (a.tris) atomicAdd((unsigned long long *)&st->tri_tests[which], a.tris);
        if (a.walks) atomicAdd((unsigned long long *)&st->packet_walks, a.walks);
        if (a.steps) atomicAdd((unsigned long long *)&st->packet_steps, a.steps);
    }
}

// warp-reduce per-thread counters into the block accumulator
__device__ __forceinline__ void acc_counters(BlockAcc &a, double mfp, double mfp_np, unsigned long long mc,
                                             unsigned long long mcnp, unsigned long long segs,
                                             unsigned long long shadow, unsigned long long contrib,
                                             unsigned long long sphere, const TravStats &ts)
{
    mfp = warp_sum_d(mfp);
    mfp_np = warp_sum_d(mfp_np);
    mc = warp_sum_u(mc);
    mcnp = warp_sum_u(mcnp);
    segs = warp_sum_u(segs);
    shadow = warp_sum_u(shadow);
    contrib = warp_sum_u(contrib);
    sphere = warp_sum_u(sphere);
    const unsigned long long nodes = warp_sum_u(ts.nodes), tris = warp_sum_u(ts.tris);
    const unsigned long long walks = warp_sum_u(ts.walks), steps = warp_sum_u(ts.steps);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&a.mfp, mfp);
        atomicAdd(&a.mfp_np, mfp_np);
        atomicAdd(&a.mfp_cnt, mc);
        atomicAdd(&a.mfp_cnt_np, mcnp);
        atomicAdd(&a.segs, segs);
        atomicAdd(&a.shadow, shadow);
        atomicAdd(&a.contrib, contrib);
        atomicAdd(&a.sphere, sphere);
        atomicAdd(&a.nodes, nodes);
        atomicAdd(&a.tris, tris);
        if (walks) atomicAdd(&a.walks, walks);
        if (steps) atomicAdd(&a.steps, steps);
    }
}

// a store pass found no slot for a reflection or record of ray rid: the host falls
// back to the counting passes if the ray is inside the waves
__device__ __forceinline__ void store_failed(const TraceWork &w, uint32_t rid)
{
    atomicMax(&w.ctr->store_fail, ~(unsigned long long)rid);
}

// slot of candidate rid among the speculative rays of a store pass, or ~0 if the
// waves are known to take it
__device__ __forceinline__ unsigned long long spec_slot(const TraceWork &w, uint32_t rid)
{
    const unsigned long long rel = (unsigned long long)rid - w.job0.first_ray;
    return rel >= w.spec_lo ? rel - w.spec_lo : ~0ull;
}

__device__ __forceinline__ void emit_record(const TraceWork &w, uint32_t key, uint32_t rid, const float *e,
                                            int B, bool store = false)
{
    const unsigned long long idx = warp_append(&w.ctr->n_records);
    if (idx < w.rec.cap) {
        w.rec.key[idx] = key;
        w.rec.rid[idx] = rid;
        float *dst = w.rec.e + idx * (unsigned long long)B;
#pragma unroll
        for (int b = 0; b < MAXB; ++b)
            if (b < B) dst[b] = e[b];
    } else if (store) {
        store_failed(w, rid);
    } else {
        raise_error(w.status, RP_ERR_CAPACITY);
    }
}

__global__ void k_setup(TraceWork w, int wave)
{
    if (wave == 0) {
        const int j = blockIdx.x * blockDim.x + threadIdx.x;
        if (j >= w.njobs) return;
        const SceneJob &J = w.jobs[j];
        JobState &s = w.js[j];
        s.wave_begin = J.first_ray;
        s.wave_count = J.num_rays;
        s.primaries = J.num_rays;
        if (J.num_rays > 0) atomicAdd((unsigned long long *)&w.stats->primaries, J.num_rays);
        if (j == 0) {
            w.stats->waves = 1;
            w.ctr->next_ray = 0;
        }
        return;
    }
    // later waves: one job, refill of the unused segment budget
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    JobState &s = w.js[0];
    const SceneJob &J = w.jobs[0];
    s.wave_begin += s.wave_count;
    const unsigned long long budget = J.num_rays * (unsigned long long)w.k.M;
    const unsigned long long used = s.segments;
    const unsigned long long unused = budget > used ? budget - used : 0ull;
    const unsigned long long count =
        (w.k.M > 0 && unused >= (unsigned long long)w.k.M) ? unused / (unsigned long long)w.k.M : 0ull;
    s.wave_count = count;
    w.ctr->next_ray = 0;
    if (count > 0) {
        w.stats->waves += 1;
        w.stats->primaries += count;
        s.primaries += count;
    }
}

// Planned refill (one job).  The waves of the segment-budget refill are sized by the
// segments of the rays before them, so traced as waves they run one after another.
// Instead passes of the paths kernel trace candidate ray ids and record each path's
// segments; k_refill_plan then finds the waves' sizes.  A store pass keeps everything
// its paths give and drops the candidates past the waves afterwards; a counting pass
// keeps only the segments, and one wave of all the waves' rays is traced after it.
// Either way the rays, paths and results are those of the waves.

// candidate rays first_ray + begin .. first_ray + begin + count for the next pass
__global__ void k_plan_block(TraceWork w, unsigned long long begin, unsigned long long count)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    w.js[0].wave_begin = w.jobs[0].first_ray + begin;
    w.js[0].wave_count = count;
    w.ctr->next_ray = 0;
}

// The waves from the candidates' segment counts: wave 1 is the N primaries; each later
// wave takes floor(unused / M) further ray ids, unused being the budget N M less the
// segments of all rays so far (as k_setup's later waves).  One block of REFILL_THREADS
// sums each wave's range; the walk resumes where the previous pass stopped.
// plan_need > 0: the waves reach past the candidates traced so far.
constexpr int REFILL_THREADS = 1024;
__global__ void __launch_bounds__(REFILL_THREADS) k_refill_plan(TraceWork w, unsigned long long cand)
{
    __shared__ unsigned long long part[REFILL_THREADS / 32];
    if (blockIdx.x != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    TraceCounters *C = w.ctr;
    const unsigned long long N = w.jobs[0].num_rays, M = (unsigned long long)w.k.M, budget = N * M;
    unsigned long long r = 0, used = 0, waves = 0, count = N, need = 0;
    if (C->plan_started) {
        r = C->plan_rays;
        used = C->plan_used;
        waves = C->plan_waves;
        count = C->plan_count;
    }
    __syncthreads();  // every thread has read the counters before thread 0 rewrites them
    while (count > 0) {  // r grows by count >= 1 each time and stays <= cand
        if (r + count > cand) {
            need = r + count;
            break;
        }
        unsigned long long seg = 0;
        const uint32_t *ps = w.plan_seg;
        unsigned long long i = r + tid;
        for (; i + 3 * REFILL_THREADS < r + count; i += 4 * REFILL_THREADS)
            seg += (unsigned long long)ps[i] + ps[i + REFILL_THREADS] + ps[i + 2 * REFILL_THREADS] +
                   ps[i + 3 * REFILL_THREADS];
        for (; i < r + count; i += REFILL_THREADS) seg += ps[i];
        for (int o = 16; o > 0; o >>= 1) seg += __shfl_xor_sync(FULL, seg, o);
        if (lane == 0) part[wid] = seg;
        __syncthreads();
        seg = 0;
        for (int q = 0; q < REFILL_THREADS / 32; ++q) seg += part[q];  // the same order in every thread
        __syncthreads();  // part is rewritten by the next wave
        used += seg;
        r += count;
        ++waves;
        const unsigned long long unused = budget > used ? budget - used : 0ull;
        count = (M > 0 && unused >= M) ? unused / M : 0ull;
    }
    if (tid == 0) {
        C->plan_need = need;
        C->plan_rays = r;
        C->plan_waves = waves;
        C->plan_used = used;
        C->plan_count = count;
        C->plan_started = 1;
    }
}

// the planned waves as one: every ray of them, with the waves' primaries and count
__global__ void k_plan_apply(TraceWork w)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    JobState &s = w.js[0];
    const SceneJob &J = w.jobs[0];
    const unsigned long long K = w.ctr->plan_rays;
    s.wave_begin = J.first_ray;
    s.wave_count = K;
    s.primaries = K;
    s.segments = 0;
    w.stats->primaries += K - J.num_rays;
    w.stats->waves = w.ctr->plan_waves;
    w.ctr->next_ray = 0;
}

// After a store pass: the statistics of its speculative candidates that the waves take
// (all of them while the waves reach past the candidates, else those before the
// waves' end), as the real pass would have added them.  A path's segments, its
// reflections (one fewer if it escaped), its path length and the part after the first
// reflection give the segment and free-path sums.
__global__ void k_spec_fold(TraceWork w, unsigned long long count)
{
    __shared__ BlockAcc acc;
    acc_init(acc);
    __syncthreads();
    const int B = w.k.B;
    const unsigned long long K = w.ctr->plan_rays;
    const unsigned long long keep =
        w.ctr->plan_need > 0 ? count : (K > w.spec_lo ? min(count, K - w.spec_lo) : 0ull);
    double mfp = 0.0, mfp_np = 0.0;
    unsigned long long mc = 0, mcnp = 0, segs = 0, sph = 0, reruns = 0;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < keep;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long h = w.plan_seg[w.spec_lo + q];
        const bool esc = w.spec.esc[q] != 0u;
        const unsigned long long hits = esc ? h - 1 : h;
        segs += h;
        mc += hits;
        if (hits > 0) {
            mcnp += hits - 1;
            mfp += w.spec.L[q];
            mfp_np += w.spec.L[q] - w.spec.t1[q];
        }
        sph += w.spec.sph[q];
        reruns += w.spec.rerun[q];
        for (int b = 0; b < B; ++b) {
            atomicAdd(esc ? &acc.esc[b] : &acc.rem[b], (double)w.spec.w[q * B + b]);
            atomicAdd(&acc.absb[b], (double)w.spec.absb[q * B + b]);
            const double late = w.spec.late[q * B + b];
            if (late != 0.0) atomicAdd(&acc.late[b], late);
        }
    }
    acc_counters(acc, mfp, mfp_np, mc, mcnp, segs, 0ull, sph, sph, TravStats{0u, 0u});
    for (int o = 16; o > 0; o >>= 1) reruns += __shfl_xor_sync(FULL, reruns, o);
    if ((threadIdx.x & 31) == 0 && reruns) atomicAdd((unsigned long long *)&w.stats->fp64_reruns, reruns);
    acc_flush(acc, w.stats, B, 0);
}

// first shadow item of every job (sum over earlier jobs of stored reflections x
// sources) and first reflection in the flattened order of the step
__device__ __forceinline__ void item_prefix(const TraceWork &w)
{
    unsigned long long acc = 0, hits = 0;
    for (int j = 0; j < w.njobs; ++j) {
        w.js[j].item_off = acc;
        w.js[j].hit_prefix = hits;
        const unsigned long long h = min(w.js[j].n_hits, w.jobs[j].hit_cap);
        acc += shadow_items(h, w.jobs[j].S);
        hits += h;
    }
    w.ctr->total_items = acc;
    w.ctr->total_hits = hits;
}

__global__ void k_item_prefix(TraceWork w)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) item_prefix(w);
}

// after the reflection order of a step with dropped rays: the job keeps the
// reflections left in the order, and its shadow items follow from those
__global__ void k_hits_kept(TraceWork w)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    w.js[0].n_hits = w.ctr->total_hits - w.ctr->dropped_hits;
    item_prefix(w);
}

// job of flattened reflection f: the last job whose first reflection is <= f
__device__ __forceinline__ int job_of_hit(const TraceWork &w, unsigned long long f)
{
    int lo = 0, hi = w.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w.js[mid].hit_prefix <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Cell of a point in its job's box with `bits` code bits: the bits go one at a time to
// the axis whose cells are then longest (ties to the lower axis), so the cells come out
// near-cubic whatever the box's proportions, and the code interleaves the axes' bits from
// the top, an axis taking part from its own highest bit on (a Morton order on unequal
// bit depths; on a cube it is the plain Morton code).
__device__ __forceinline__ uint32_t cell_code(const SceneView &sc, float3 p, int bits)
{
    int nb[3] = {0, 0, 0};
    float ce[3] = {fmaxf(sc.ext[0], 0.f), fmaxf(sc.ext[1], 0.f), fmaxf(sc.ext[2], 0.f)};
    for (int i = 0; i < bits; ++i) {
        const int a = (ce[0] >= ce[1] && ce[0] >= ce[2]) ? 0 : (ce[1] >= ce[2] ? 1 : 2);
        ++nb[a];
        ce[a] *= 0.5f;
    }
    const float pc[3] = {p.x, p.y, p.z};
    uint32_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float n = (float)(1u << nb[a]);
        const float e = sc.ext[a] > 0.f ? sc.ext[a] : 1.f;
        q[a] = (uint32_t)fminf(fmaxf((pc[a] - sc.lo[a]) / e * n, 0.f), n - 1.f);
    }
    const int top = max(nb[0], max(nb[1], nb[2]));
    uint32_t code = 0;
    for (int i = top - 1; i >= 0; --i) {
#pragma unroll
        for (int a = 2; a >= 0; --a)
            if (i < nb[a]) code = (code << 1) | ((q[a] >> i) & 1u);
    }
    return code;
}

constexpr uint32_t DROPPED_CELL = 0xffffffffu;

// cell of every stored reflection, and the cell counts
__global__ void k_hit_cells(TraceWork w)
{
    const unsigned long long n = w.ctr->total_hits;
    const int bits = w.horder.bits;
    for (unsigned long long f = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; f < n;
         f += (unsigned long long)gridDim.x * blockDim.x) {
        const int job = w.njobs > 1 ? job_of_hit(w, f) : 0;
        const SceneJob &J = w.njobs > 1 ? w.jobs[job] : w.job0;
        const unsigned long long slot = J.hit_off + (f - (w.njobs > 1 ? w.js[job].hit_prefix : 0ull));
        if (!RP_IN_RANGE(slot, w.hits.cap, w.status) || !RP_IN_RANGE(f, w.hits.cap, w.status)) continue;
        if (w.rid_end && (unsigned long long)w.hits.rid[slot] >= w.rid_end) {
            w.horder.cell[f] = DROPPED_CELL;  // a ray past the waves of a store pass
            atomicAdd(&w.ctr->dropped_hits, 1ull);
            continue;
        }
        const float4 P = w.hits.p[slot];
        const uint32_t cell = ((uint32_t)job << bits) | cell_code(J.sc, xyz(P), bits);
        if (!RP_IN_RANGE(cell, w.horder.ncells, w.status)) continue;
        w.horder.cell[f] = cell;
        atomicAdd(&w.horder.cnt[cell], 1u);
    }
}

// reflection slots in cell order (the order inside a cell is not fixed)
__global__ void k_hit_scatter(TraceWork w)
{
    const unsigned long long n = w.ctr->total_hits;
    for (unsigned long long f = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; f < n;
         f += (unsigned long long)gridDim.x * blockDim.x) {
        const int job = w.njobs > 1 ? job_of_hit(w, f) : 0;
        const SceneJob &J = w.njobs > 1 ? w.jobs[job] : w.job0;
        const unsigned long long slot = J.hit_off + (f - (w.njobs > 1 ? w.js[job].hit_prefix : 0ull));
        if (w.horder.cell[f] == DROPPED_CELL) continue;
        if (!RP_IN_RANGE(w.horder.cell[f], w.horder.ncells, w.status)) continue;
        const uint32_t pos = atomicAdd(&w.horder.cnt[w.horder.cell[f]], 1u);
        if (RP_IN_RANGE(pos, w.hits.cap, w.status)) w.horder.perm[pos] = (uint32_t)slot;
    }
}

// copy of the records the shadow rays read, in cell order (random reads, coalesced writes)
__global__ void k_hit_gather(TraceWork w)
{
    const unsigned long long n = w.ctr->total_hits;
    const int B = w.k.B;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long slot = w.horder.perm[i];
        if (!RP_IN_RANGE(slot, w.hits.cap, w.status) || !RP_IN_RANGE(i, w.shits.cap, w.status)) continue;
        w.shits.p[i] = w.hits.p[slot];
        w.shits.n[i] = w.hits.n[slot];
        w.shits.rid[i] = w.hits.rid[slot];
        const float *src = w.hits.ws + slot * B;
        float *dst = w.shits.ws + i * B;
        for (int b = 0; b < B; ++b) dst[b] = src[b];
    }
}

// job of shadow item q: the last job whose first item is <= q
__device__ __forceinline__ int job_of_item(const TraceWork &w, unsigned long long q)
{
    int lo = 0, hi = w.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w.js[mid].item_off <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Warp-aggregated append on a per-job counter: lanes grouped by job.
__device__ __forceinline__ unsigned long long warp_append_job(unsigned long long *counter, int job)
{
    const unsigned mask = __activemask();
    const unsigned peers = __match_any_sync(mask, job);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + (unsigned long long)__popc(peers & ((1u << lane) - 1u));
}

// closest-hit segments of a single-job step, for the next wave's refill
__device__ __forceinline__ void wave_segments_flush(const TraceWork &w, unsigned long long segs)
{
    for (int o = 16; o > 0; o >>= 1) segs += __shfl_xor_sync(FULL, segs, o);
    if ((threadIdx.x & 31) == 0 && segs) atomicAdd(&w.js[0].segments, segs);
}

// Path state in precision R.  The default carries the origin, direction and path
// length of each path in FP64 while BVH traversal and the triangle choice stay in
// FP32: the hit distance is re-computed in FP64 on the chosen triangle, so that a
// path keeps FP64 accuracy over many reflections (in FP32 the position error grows
// with every oblique reflection until late reflections pick different triangles).
// With RP_FLAG_FP32_PATHS the whole path is FP32.
template <typename R>
struct V3 {
    R x, y, z;
    // hidden friends: found by argument-dependent lookup only, so they do not hide
    // the float3 operators of the enclosing namespace
    friend __device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
    friend __device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
    friend __device__ __forceinline__ V3 operator*(V3 a, R s) { return {a.x * s, a.y * s, a.z * s}; }
};
template <typename R>
__device__ __forceinline__ V3<R> v3(R x, R y, R z)
{
    return {x, y, z};
}
template <typename R>
__device__ __forceinline__ R dot3(V3<R> a, V3<R> b)
{
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename R>
__device__ __forceinline__ V3<R> cross3(V3<R> a, V3<R> b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R>
__device__ __forceinline__ V3<R> from4(float4 v)
{
    return {(R)v.x, (R)v.y, (R)v.z};
}
template <typename R>
__device__ __forceinline__ float3 to_f3(V3<R> v)
{
    return mk3((float)v.x, (float)v.y, (float)v.z);
}
__device__ __forceinline__ void sincospi_r(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_r(double x, double *s, double *c) { sincospi(x, s, c); }
template <typename R>
__device__ __forceinline__ R u01r(uint32_t x)
{
    return (R)(x >> 8) * (R)(1.0 / 16777216.0);
}

template <typename R>
__device__ __forceinline__ V3<R> primary_dir_r(uint32_t rid, uint32_t scene_id, uint32_t k0, uint32_t k1)
{
    const U4 r = philox4x32_10(rid, scene_id, 0u, 0u, k0, k1);
    const R z = (R)1 - (R)2 * u01r<R>(r.x);
    const R rad = sqrt(max((R)0, (R)1 - z * z));
    R s, c;
    sincospi_r((R)2 * u01r<R>(r.y), &s, &c);
    return v3<R>(rad * c, rad * s, z);
}

// STORE: a store pass of the planned refill (one job, FP64 paths): everything of the
// real pass, with the statistics of speculative candidates kept per ray (SpecRays)
template <typename R, bool HASH, bool COUNT, bool BATCH, bool STORE = false>
__global__ void __launch_bounds__(PATH_THREADS, 4) k_paths(TraceWork w)
{
    __shared__ int sstack[SMEM_STACK * PATH_THREADS];
    __shared__ BlockAcc acc;
    acc_init(acc);
    __syncthreads();

    const TraceConsts &k = w.k;
    const int B = k.B, T = k.T, M = k.M;
    const int lane = threadIdx.x & 31;
    const unsigned long long seed = w.seed ? w.seed[0] : w.seed_val;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const unsigned long long wave_begin = BATCH ? 0ull : w.js[0].wave_begin;  // set by k_setup
    const unsigned long long wave_count = BATCH ? 0ull : w.js[0].wave_count;
    const unsigned long long vtotal = BATCH ? (unsigned long long)w.nchunks * w.chunk_rays : wave_count;
    const float inv_pi_rs2 = 1.0f / (PI_F * k.rs * k.rs);
    const bool plan = !BATCH && !STORE && w.plan;  // count each path's segments only (planned refill)

    double mfp_np = 0.0;
    unsigned long long mcnp = 0, sphere = 0, contrib = 0, reruns = 0, segs_all = 0, mc_all = 0;
    double mfp_all = 0.0;
    TravStats ts = {0u, 0u};

    // path state
    bool have = false, done = vtotal == 0;
    int job = 0;
    uint32_t rid = 0;
    V3<R> o = v3<R>(0, 0, 0), d = o;
    R L = 0;
    // the path's band weights and absorbed weights, in the lane's own column of shared
    // memory (band b at [b * PATH_THREADS], no bank conflicts): in registers they made
    // the kernel spill at its 128-register bound
    __shared__ float swgt[MAXB][PATH_THREADS], sabs[MAXB][PATH_THREADS];
    float *const wgt = &swgt[0][threadIdx.x];
    float *const absorbed = &sabs[0][threadIdx.x];
    int prev = -1, h = 1;
    bool spec_prev = false;
    uint64_t hash = FNV_OFFSET;

    while (true) {
        const unsigned need = __ballot_sync(FULL, !have && !done);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&w.ctr->next_ray, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (!have && !done) {
                const unsigned long long v = base + __popc(need & ((1u << lane) - 1u));
                bool got = false;
                if (v >= vtotal) {
                    done = true;
                } else if (BATCH) {
                    const RayChunk ch = w.chunks[v / (unsigned long long)w.chunk_rays];
                    const unsigned r = (unsigned)(v % (unsigned long long)w.chunk_rays);
                    if (r < (unsigned)ch.count) {  // otherwise padding of a short chunk
                        job = ch.job;
                        rid = (uint32_t)(ch.start + r);
                        got = true;
                    }
                } else {
                    rid = (uint32_t)(wave_begin + v);
                    got = true;
                }
                if (got) {
                    const SceneJob &J = BATCH ? w.jobs[job] : w.job0;
                    have = true;
                    o = from4<R>(__ldg(w.pos + J.lis));
                    d = primary_dir_r<R>(rid, J.scene_id, key0, key1);
                    L = 0;
#pragma unroll
                    for (int b = 0; b < MAXB; ++b) {
                        wgt[b * PATH_THREADS] = 1.0f;
                        absorbed[b * PATH_THREADS] = 0.0f;
                    }
                    prev = -1;
                    h = 1;
                    spec_prev = false;
                    hash = FNV_OFFSET;
                }
            }
        }
        if (!__any_sync(FULL, have) && __all_sync(FULL, done || have)) break;
        if (!have) continue;

        const SceneJob &J = BATCH ? w.jobs[job] : w.job0;
        const SceneView &sc = J.sc;
        // ---- one segment: closest hit (FP32 traversal) ----
        const float3 of = to_f3(o), df = to_f3(d);
        const float Lf = (float)L;
        float tf;
        bool amb = false, exact = false;
        int tri;
        R t_exact = 0;
        if (sizeof(R) == 8) {
            tri = traverse<false, COUNT, true>(sc, of, df, sc.tmin, INFINITY, prev, sstack + threadIdx.x, tf, ts,
                                               w.status, &amb);
            if (amb) {
                // the FP32 answer may depend on rounding: decide it in FP64
                double te;
                tri = traverse_exact<false>(sc, D3{(double)o.x, (double)o.y, (double)o.z},
                                            D3{(double)d.x, (double)d.y, (double)d.z}, sc.tmin_d, INFINITY, prev,
                                            sstack + threadIdx.x, te, w.status);
                exact = true;
                t_exact = (R)te;
                tf = (float)te;
                const unsigned long long q = STORE ? spec_slot(w, rid) : ~0ull;
                if (q != ~0ull) ++w.spec.rerun[q];
                else ++reruns;
            }
        } else {
            tri = traverse<false, COUNT, false>(sc, of, df, sc.tmin, INFINITY, prev, sstack + threadIdx.x, tf, ts,
                                                w.status);
        }
        if (!STORE || spec_slot(w, rid) == ~0ull) ++segs_all;
        if (!plan && spec_prev && h - 1 >= k.min_order) {
            // the job's sources as spheres of radius r_s, seen through the specular bounce
            for (int s = 0; s < J.S; ++s) {
                const int gs = J.src_off + s;
                const float4 cs = __ldg(w.pos + gs);
                const float3 oc = of - xyz(cs);
                const float bq = dot(oc, df);
                const float cq = dot(oc, oc) - k.rs * k.rs;
                const float disc = bq * bq - cq;
                if (disc < 0.f) continue;
                const float tsph = -bq - sqrtf(disc);
                if (!(tsph > sc.tmin) || (tri >= 0 && !(tsph < tf))) continue;
                const unsigned long long q = STORE ? spec_slot(w, rid) : ~0ull;
                if (q != ~0ull) {
                    ++w.spec.sph[q];
                } else {
                    ++sphere;
                    ++contrib;
                }
                float e[MAXB];
#pragma unroll
                for (int b = 0; b < MAXB; ++b) e[b] = wgt[b * PATH_THREADS] * inv_pi_rs2;
                float binf;
                const float x = ((Lf + tsph) / k.c) * k.rate;
                if (fabsf(x - rintf(x)) < BIN_GUARD) {
                    // close to a bin boundary: decide with the path-precision state
                    const V3<R> oc2 = o - from4<R>(cs);
                    const R b2 = dot3(oc2, d);
                    const R c2 = dot3(oc2, oc2) - (R)k.rs * (R)k.rs;
                    const R t2 = -b2 - sqrt(max((R)0, b2 * b2 - c2));
                    binf = (float)floor(((L + t2) / (R)k.c) * (R)k.rate);
                } else {
                    binf = floorf(x);
                }
                if (binf < (float)T) {
                    emit_record(w, (uint32_t)(gs - w.src_base) * (uint32_t)T + (uint32_t)binf, rid, e, B, STORE);
                } else if (q != ~0ull) {
                    for (int b = 0; b < B; ++b) w.spec.late[q * B + b] += (double)e[b];
                } else {
#pragma unroll
                    for (int b = 0; b < MAXB; ++b)
                        if (b < B) atomicAdd(&acc.late[b], (double)e[b]);
                }
            }
        }
        if (HASH) {
            const uint32_t v = tri < 0 ? 0xffffffffu : __float_as_uint(__ldg(sc.tris + 3 * tri + 1).w);
            hash = fnv_u32(hash, v);
        }
        bool end_ray = false;
        if (tri < 0) {
            if (!STORE || spec_slot(w, rid) == ~0ull) {
#pragma unroll
                for (int b = 0; b < MAXB; ++b)
                    if (b < B) atomicAdd(&acc.esc[b], (double)wgt[b * PATH_THREADS]);
            }
            end_ray = true;
        } else {
            const float4 ta = __ldg(sc.tris + 3 * tri), tb = __ldg(sc.tris + 3 * tri + 1),
                         tc = __ldg(sc.tris + 3 * tri + 2);
            const V3<R> v0 = from4<R>(ta), e1 = from4<R>(tb) - v0, e2 = from4<R>(tc) - v0;
            // hit distance on the chosen triangle in the path precision
            R t = exact ? t_exact : (R)tf;
            if (sizeof(R) == 8 && !exact) {
                const V3<R> pv = cross3(d, e2);
                const R det = dot3(e1, pv);
                if (det != (R)0) t = dot3(e2, cross3(o - v0, e1)) / det;
            }
            L += t;
            const V3<R> p = o + d * t;
            const unsigned long long qs = STORE ? spec_slot(w, rid) : ~0ull;
            if (qs != ~0ull) {
                if (h == 1) w.spec.t1[qs] = (double)t;
            } else {
                mfp_all += (double)t;
                ++mc_all;
                if (h > 1) {
                    mfp_np += (double)t;
                    ++mcnp;
                }
            }
            V3<R> n = cross3(e1, e2);
            n = n * ((R)1 / sqrt(dot3(n, n)));
            if (dot3(n, d) > (R)0) n = n * (R)-1;
            const int mat = __float_as_int(ta.w);
            const float *al = sc.alpha + mat * B;
#pragma unroll
            for (int b = 0; b < MAXB; ++b) {
                if (b < B) {
                    const float a = __ldg(al + b);
                    absorbed[b * PATH_THREADS] += wgt[b * PATH_THREADS] * a;
                    wgt[b * PATH_THREADS] *= (1.0f - a);
                }
            }
            // an early reflection (below min_order, order <= 2) is kept apart for the
            // early-path cache when the step asks for it (rp_trace_er)
            const bool early = !BATCH && w.er.cap > 0 && h < k.min_order && h <= 2;
            if (!plan && (h >= k.min_order || early) && J.S > 0) {
                const Hits &dst = early ? w.er.hits : w.hits;
                const unsigned long long cap = early ? w.er.cap : J.hit_cap, off = early ? 0ull : J.hit_off;
                const unsigned long long jl =
                    early ? warp_append(&w.ctr->n_er)
                          : (BATCH ? warp_append_job(&w.js[job].n_hits, job) : warp_append(&w.js[0].n_hits));
                if (jl < cap && RP_IN_RANGE(off + jl, dst.cap, w.status)) {
                    const unsigned long long j = off + jl;
                    const float4 phi = make_float4((float)p.x, (float)p.y, (float)p.z, (float)L);
                    dst.p[j] = phi;
                    dst.plo[j] = make_float4((float)(p.x - (R)phi.x), (float)(p.y - (R)phi.y),
                                             (float)(p.z - (R)phi.z), (float)(L - (R)phi.w));
                    dst.n[j] = make_float4((float)n.x, (float)n.y, (float)n.z, __int_as_float(tri));
                    const float *sb = sc.scat + mat * B;
#pragma unroll
                    for (int b = 0; b < MAXB; ++b)
                        if (b < B) dst.ws[j * B + b] = wgt[b * PATH_THREADS] * __ldg(sb + b);
                    dst.rid[j] = rid;
                    if (early) w.er.prev[j] = prev;
                } else if (STORE) {
                    store_failed(w, rid);
                } else {
                    raise_error(w.status, RP_ERR_CAPACITY);
                }
            }
            if (h == M) {
                if (!STORE || spec_slot(w, rid) == ~0ull) {
#pragma unroll
                    for (int b = 0; b < MAXB; ++b)
                        if (b < B) atomicAdd(&acc.rem[b], (double)wgt[b * PATH_THREADS]);
                }
                end_ray = true;
            } else {
                const U4 r = philox4x32_10(rid, J.scene_id, (uint32_t)h, 0u, key0, key1);
                if ((r.z >> 8) < __ldg(sc.thr + mat)) {
                    // cosine-weighted hemisphere about n (Malley), frame of Duff et al. 2017
                    const R u0 = u01r<R>(r.x), u1 = u01r<R>(r.y);
                    const R rr = sqrt(u1);
                    R sn, cn;
                    sincospi_r((R)2 * u0, &sn, &cn);
                    const R lx = rr * cn, ly = rr * sn, lz = sqrt(max((R)0, (R)1 - u1));
                    const R sg = n.z >= (R)0 ? (R)1 : (R)-1;
                    const R aa = (R)-1 / (sg + n.z);
                    const R bb = n.x * n.y * aa;
                    const V3<R> b1 = v3<R>((R)1 + sg * n.x * n.x * aa, sg * bb, -sg * n.x);
                    const V3<R> b2 = v3<R>(bb, sg + n.y * n.y * aa, -n.y);
                    d = b1 * lx + b2 * ly + n * lz;
                    const float *wd = sc.wdiff + mat * B;
#pragma unroll
                    for (int b = 0; b < MAXB; ++b)
                        if (b < B) wgt[b * PATH_THREADS] *= __ldg(wd + b);
                    spec_prev = false;
                } else {
                    d = d - n * ((R)2 * dot3(d, n));
                    d = d * ((R)1 / sqrt(dot3(d, d)));
                    const float *wsp = sc.wspec + mat * B;
#pragma unroll
                    for (int b = 0; b < MAXB; ++b)
                        if (b < B) wgt[b * PATH_THREADS] *= __ldg(wsp + b);
                    spec_prev = true;
                }
                o = p;
                prev = tri;
                ++h;
            }
        }
        if (end_ray) {
            const unsigned long long q = STORE ? spec_slot(w, rid) : ~0ull;
            if (q != ~0ull) {
                // the speculative ray's end: band weights, absorbed weights, path length
                for (int b = 0; b < B; ++b) {
                    w.spec.w[q * B + b] = wgt[b * PATH_THREADS];
                    w.spec.absb[q * B + b] = absorbed[b * PATH_THREADS];
                }
                w.spec.L[q] = (double)L;
                w.spec.esc[q] = tri < 0 ? 1u : 0u;
            } else {
#pragma unroll
                for (int b = 0; b < MAXB; ++b)
                    if (b < B) atomicAdd(&acc.absb[b], (double)absorbed[b * PATH_THREADS]);
            }
            if (HASH && w.ray_hash && rid >= J.first_ray && rid - J.first_ray < J.num_rays)
                w.ray_hash[rid - J.first_ray] = hash;
            if ((plan || STORE) && RP_IN_RANGE(rid - J.first_ray, J.num_rays * (unsigned long long)M, w.status))
                w.plan_seg[rid - J.first_ray] = (uint32_t)h;  // the path's segments
            have = false;
        }
    }
    if (plan) return;  // the counting pass leaves the statistics to the real one
    if (!BATCH) wave_segments_flush(w, segs_all);
    acc_counters(acc, mfp_all, mfp_np, mc_all, mcnp, segs_all, 0ull, contrib, sphere, ts);
    for (int o = 16; o > 0; o >>= 1) reruns += __shfl_xor_sync(FULL, reruns, o);
    if (lane == 0 && reruns) atomicAdd((unsigned long long *)&w.stats->fp64_reruns, reruns);
    acc_flush(acc, w.stats, B, 0);
}

// Emit the contribution of a visible (reflection j, global source gs) pair: energy
// w_b s_b cos(theta) / (pi d^2), arrival (L + d) / c.  An FP32 arrival time that
// lands within BIN_GUARD of a bin boundary is re-decided in FP64 from the stored
// residuals.
__device__ __forceinline__ void shadow_contribution(const TraceWork &w, BlockAcc &acc, unsigned long long j, int gs,
                                                    float f, float dist)
{
    const TraceConsts &k = w.k;
    const int B = k.B, T = k.T;
    if (!RP_IN_RANGE(j, w.shits.cap, w.status) || !RP_IN_RANGE(w.horder.perm[j], w.hits.cap, w.status)) return;
    const float4 P = w.shits.p[j];
    float e[MAXB];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) e[b] = b < B ? w.shits.ws[j * B + b] * f : 0.f;
    float binf;
    const float x = ((P.w + dist) / k.c) * k.rate;
    if (fabsf(x - rintf(x)) < BIN_GUARD) {
        const float4 lo = w.hits.plo[w.horder.perm[j]];
        const float4 cs = __ldg(w.pos + gs);
        const double dx = (double)cs.x - ((double)P.x + (double)lo.x);
        const double dy = (double)cs.y - ((double)P.y + (double)lo.y);
        const double dz = (double)cs.z - ((double)P.z + (double)lo.z);
        const double dd = sqrt(dx * dx + dy * dy + dz * dz);
        const double tt = ((double)P.w + (double)lo.w + dd) / (double)k.c;
        binf = (float)floor(tt * (double)k.rate);
    } else {
        binf = floorf(x);
    }
    if (binf < (float)T) {
        emit_record(w, (uint32_t)(gs - w.src_base) * (uint32_t)T + (uint32_t)binf, w.shits.rid[j], e, B);
    } else {
#pragma unroll
        for (int b = 0; b < MAXB; ++b)
            if (b < B) atomicAdd(&acc.late[b], (double)e[b]);
    }
}

// (reflection in the cell-ordered copy, global source) of shadow item q of job `job`;
// false for a hole.  A job's items come in tiles of 32 reflections (consecutive in
// cell order) x its S sources; the tiles go in groups of SHADOW_TILE_GROUP, source-major
// inside a group: each run of 32 items is rays from nearby points to one source, and
// consecutive runs are neighbouring tiles towards the same source.  The last tile of a
// job may hold fewer than 32 reflections; its runs keep 32 slots and the slots past its
// reflections are holes, so that every job's items and every run start at a multiple of
// 32 and a warp's 32 consecutive items are one run.
__device__ __forceinline__ bool item_slot(const TraceWork &w, bool batch, int job, unsigned long long q,
                                          unsigned long long &j, int &gs)
{
    const SceneJob &J = batch ? w.jobs[job] : w.job0;
    const JobState &js = w.js[job];
    const unsigned long long local = q - (batch ? js.item_off : 0ull);
    const unsigned long long n = min(js.n_hits, J.hit_cap);
    // run of 32 items: group of SHADOW_TILE_GROUP tiles, then source, then tile in the group
    const unsigned long long run = local >> 5;
    const unsigned long long gS = (unsigned long long)SHADOW_TILE_GROUP * (unsigned long long)J.S;
    const unsigned long long ntiles = (n + 31ull) / 32ull;
    unsigned long long grp, within, src, gc;
    if (run < 0x100000000ull) {  // 32-bit divisions (64-bit ones are long instruction sequences)
        grp = (uint32_t)run / (uint32_t)gS;  // gS <= 32 x RP_MAX_SOURCES
        within = run - grp * gS;
        gc = ntiles > grp * SHADOW_TILE_GROUP ? min((unsigned long long)SHADOW_TILE_GROUP, ntiles - grp * SHADOW_TILE_GROUP)
                                              : 1ull;  // tiles in this group
        src = (uint32_t)within / (uint32_t)gc;
    } else {
        grp = run / gS;
        within = run - grp * gS;
        gc = ntiles > grp * SHADOW_TILE_GROUP ? min((unsigned long long)SHADOW_TILE_GROUP, ntiles - grp * SHADOW_TILE_GROUP)
                                              : 1ull;
        src = within / gc;
    }
    const unsigned long long tile = grp * SHADOW_TILE_GROUP + (within - src * gc);
    const unsigned r = (unsigned)(local & 31u);
    j = js.hit_prefix + tile * 32ull + r;
    gs = J.src_off + (int)src;
    const bool real = tile * 32ull + r < n;
    return real && RP_IN_RANGE(j, w.shits.cap, w.status);
}

// (job, reflection, global source) of shadow item q; false for a hole
__device__ __forceinline__ bool item_target(const TraceWork &w, bool batch, unsigned long long q, int &job,
                                            unsigned long long &j, int &gs)
{
    job = batch ? job_of_item(w, q) : 0;
    return item_slot(w, batch, job, q, j, gs);
}

// job of item q, given a job `from` whose first item is <= q (items of later jobs
// follow in job order)
__device__ __forceinline__ int job_from(const TraceWork &w, int from, unsigned long long q)
{
    while (from + 1 < w.njobs && w.js[from + 1].item_off <= q) ++from;
    return from;
}

// Shadow rays of one chunk of the step's items q = (reflection, source) pairs,
// reflection-major within each job.  Persistent threads with per-lane refill:
// each lane advances its any-hit query a few nodes at a time and takes the next
// item as soon as its query ends, so lanes of a warp do not idle behind the longest
// ray.  Queries whose FP32 answer is rounding-sensitive are queued for the FP64
// kernel below (EXACT); when the queue is full the FP32 answer stands.
template <bool COUNT, bool EXACT, bool BATCH>
__global__ void __launch_bounds__(SHADOW_THREADS, 7) k_shadow(TraceWork w, unsigned long long chunk)
{
    const unsigned long long total = w.ctr->total_items;
    const unsigned long long q0 = chunk * w.items_per_chunk;
    const unsigned long long items = total > q0 ? min(w.items_per_chunk, total - q0) : 0ull;
    if (items == 0) return;  // a record chunk past the step's items (the whole block)
    __shared__ int sstack[SMEM_STACK * SHADOW_THREADS];
    __shared__ BlockAcc acc;
    acc_init(acc);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int steps_per_visit = w.shadow_steps;
    const float inv_pi = 1.0f / PI_F;
    int lstack[LOCAL_STACK];

    unsigned long long shadow = 0, contrib = 0;
    TravStats ts = {0u, 0u};
    bool busy = false, exhausted = items == 0;
    unsigned long long item = 0;
    int job = 0;
    AnyRay ray;
    float3 dir = mk3(0.f, 0.f, 0.f);
    AnyState st = {-1, 0, INFINITY, false, false};
    int steps = 0, iter_cap = 0;
    float f = 0.f, dist = 0.f;
    unsigned long long win = 0, win_end = 0;  // the warp's window of items (warp-uniform)
    while (true) {
        unsigned need = __ballot_sync(FULL, !busy && !exhausted);
        while (need) {
            if (win >= win_end) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(&w.ctr->next_item, (unsigned long long)SHADOW_WINDOW);
                b = __shfl_sync(FULL, b, 0);
                if (b >= items) {
                    if ((need >> lane) & 1u) exhausted = true;
                    break;
                }
                win = b;
                win_end = min(b + (unsigned long long)SHADOW_WINDOW, items);
            }
            const unsigned avail = (unsigned)min(win_end - win, 32ull);
            const unsigned rank = __popc(need & ((1u << lane) - 1u));
            if (((need >> lane) & 1u) && rank < avail) {
                {
                    const unsigned long long my = win + rank;
                    item = q0 + my;
                    unsigned long long j;
                    int gs;
                    const bool real = item_target(w, BATCH, item, job, j, gs);
                    const SceneView &sc = BATCH ? w.jobs[job].sc : w.job0.sc;
                    const float4 P = real ? w.shits.p[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 N = real ? w.shits.n[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float3 p = xyz(P);
                    const float3 v = xyz(__ldg(w.pos + gs)) - p;
                    const float dist2 = dot(v, v);
                    dist = sqrtf(dist2);
                    const float cth = dot(xyz(N), v) / dist;
                    if (real && cth > 0.f) {
                        ++shadow;
                        dir = v * (1.0f / dist);
                        ray = make_any_ray(p, dir, sc.tmin, dist, __float_as_int(N.w));
                        st = {0, 0, INFINITY, false, false};
                        steps = 0;
                        iter_cap = sc.iter_cap;
                        f = cth * inv_pi / dist2;
                        busy = true;
                    }
                }
            }
            win += min(avail, (unsigned)__popc(need));
            need = __ballot_sync(FULL, !busy && !exhausted);
        }
        if (__all_sync(FULL, !busy && exhausted)) break;
        if (!busy) continue;
        const SceneView &sc = BATCH ? w.jobs[job].sc : w.job0.sc;
        bool done = any_hit_steps<COUNT, EXACT>(sc, ray, dir, st, sstack + threadIdx.x, lstack, steps_per_visit, ts,
                                                 w.status);
        steps += steps_per_visit;
        if (!done && steps > iter_cap) {
            raise_error(w.status, RP_ERR_TIMEOUT);
            done = true;
        }
        if (!done) continue;
        busy = false;
        const bool amb = EXACT && !st.clear && st.amb_t < INFINITY;
        if (amb) {
            const unsigned long long r = warp_append(&w.ctr->n_rerun);
            if (r < w.rerun_cap) {
                w.rerun[r] = item;
                continue;
            }
        }
        if (!st.blocked) {
            unsigned long long j;
            int gs;
            item_slot(w, BATCH, job, item, j, gs);
            ++contrib;
            shadow_contribution(w, acc, j, gs, f, dist);
        }
    }
    acc_counters(acc, 0.0, 0.0, 0ull, 0ull, 0ull, shadow, contrib, 0ull, ts);
    acc_flush(acc, w.stats, w.k.B, 1);
}

// the vector from reflection j (cell-ordered copy) to global source gs, its squared length
// and the cosine at the reflection; the packet kernel decides with it whether an item
// needs a ray, and again when it sets the ray up (the same instructions, the same answer)
__device__ __forceinline__ void shadow_geometry(const TraceWork &w, unsigned long long j, int gs, float3 &v,
                                                float &dist2, float &cth)
{
    const float4 P = w.shits.p[j];
    const float4 N = w.shits.n[j];
    v = xyz(__ldg(w.pos + gs)) - xyz(P);
    dist2 = dot(v, v);
    cth = dot(xyz(N), v) / sqrtf(dist2);
}

// Shadow rays as packets.  A packet is 32 consecutive items -- in the cell-ordered
// tiles, rays from nearby points towards one source -- that walk the BVH together: one
// node fetch per warp, and a stack of the warp's own in shared memory whose entries
// carry the mask of lanes whose ray reached the node.  A lane tests only the nodes its
// own ray reaches and leaves the walk once it has a clear blocker, so its answer is the
// single-ray answer of any_hit_steps.  Items of different jobs in one packet walk their
// own BVHs one after the other.
// A warp takes up to SHADOW_TILE_GROUP packets at a time: neighbouring tiles towards one
// source.  Rays from neighbouring points to the same source are mostly blocked by the
// same few triangles, so each packet first walks the subtree where the warp's previous
// packet found a blocker (SHADOW_HINT_UP levels above that leaf; for a group's first
// packet, the latest hint any warp left for the source, else the region around the
// source), and only the lanes still without an answer then walk the whole tree.  Which
// triangles are tested first changes the work, not the answers.
template <bool COUNT, bool EXACT, bool BATCH>
__global__ void __launch_bounds__(SHADOW_THREADS, 7) k_shadow_packet(TraceWork w, unsigned long long chunk)
{
    const unsigned long long total = w.ctr->total_items;
    const unsigned long long q0 = chunk * w.items_per_chunk;
    const unsigned long long items = total > q0 ? min(w.items_per_chunk, total - q0) : 0ull;
    if (items == 0) return;  // a record chunk past the step's items (the whole block)
    __shared__ int pnode[SHADOW_THREADS / 32][STACK_DEPTH];
    __shared__ unsigned pmask[SHADOW_THREADS / 32][STACK_DEPTH];
    __shared__ uint32_t pqueue[SHADOW_THREADS / 32][64];  // the warp's items to trace (offsets in the chunk)
    __shared__ BlockAcc acc;
    acc_init(acc);
    __syncthreads();

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float inv_pi = 1.0f / PI_F;
    unsigned long long shadow = 0, contrib = 0;
    TravStats ts = {0u, 0u};
    int *const sn = pnode[wid];
    unsigned *const sm = pmask[wid];

    // where the warp's last packet towards source hint_gs found a blocker: the node
    // SHADOW_HINT_UP levels above that leaf (0: none).  The next packet towards the same
    // source starts there.
    int hint = 0, hint_gs = -1;
    // packets per fetch: a whole group of tiles when every warp gets several, fewer on
    // small problems so that they still spread over the GPU
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x / 32);
    const int per_fetch = (int)max(1ull, min((unsigned long long)SHADOW_TILE_GROUP, items / (64ull * warps)));
    uint32_t *const queue = pqueue[wid];
    // a chunk's items fit 32 bits (a chunk holds at most the record budget's items)
    if (items >= 0xffffff00ull) {
        if (threadIdx.x == 0 && blockIdx.x == 0) raise_error(w.status, RP_ERR_INVALID_ARG);
        return;
    }
    while (true) {
        unsigned long long blk64 = 0;
        if (lane == 0) blk64 = atomicAdd(&w.ctr->next_item, 32ull * per_fetch);
        blk64 = __shfl_sync(FULL, blk64, 0);
        if (blk64 >= items) break;
        // The block's items whose reflection faces the source go through the warp's queue, and
        // packets are made of 32 of them at a time: a packet's lanes all carry a ray.
        const uint32_t bend = (uint32_t)min(blk64 + 32ull * per_fetch, items);
        uint32_t cur = (uint32_t)blk64;
        int nq = 0;        // queued items (warp-uniform)
        bool first = true;  // the block's first packet
        while (true) {
            while (nq < 32 && cur < bend) {
                const uint32_t it = cur + lane;
                bool want = false;
                if (it < bend) {
                    const int jb = BATCH ? job_of_item(w, q0 + it) : 0;
                    unsigned long long j;
                    int gs;
                    const bool real = item_slot(w, BATCH, jb, q0 + it, j, gs);
                    float3 v;
                    float dist2, cth;
                    if (real) shadow_geometry(w, j, gs, v, dist2, cth);
                    want = real && cth > 0.f;
                }
                const unsigned bal = __ballot_sync(FULL, want);
                if (want) queue[nq + __popc(bal & ((1u << lane) - 1u))] = it;  // < 63
                nq += __popc(bal);
                cur += 32;
            }
            if (nq == 0) break;
            __syncwarp();
            const int take = min(nq, 32);
            const bool has = lane < take;
            const uint32_t b0 = has ? queue[lane] : 0u;
            __syncwarp();
            if (nq > 32 && lane < nq - 32) queue[lane] = queue[32 + lane];  // the rest to the front
            __syncwarp();
            nq -= take;
            const unsigned long long item = q0 + b0;
            bool traced = false;  // this lane traces a shadow ray
            // the job of the packet's first item (warp-uniform), then each lane's own
            int job = BATCH ? job_of_item(w, q0 + __shfl_sync(FULL, b0, 0)) : 0;
            AnyRay ray;
            float3 dir = mk3(0.f, 0.f, 0.f);
            float f = 0.f, dist = 0.f;
            AnyState st = {-1, 0, INFINITY, false, false};
            int start = 0;   // the region around the lane's source
            int my_gs = -1;  // the lane's source
            int blk_leaf = -1;  // the leaf whose triangle blocked this lane's ray
            if (has) {
                unsigned long long j;
                int gs;
                if (BATCH) job = job_from(w, job, item);
                const bool real = item_slot(w, BATCH, job, item, j, gs);
                my_gs = gs;
                if (w.src_node) start = w.src_node[gs];
                const SceneView &sc = BATCH ? w.jobs[job].sc : w.job0.sc;
                float3 v;
                float dist2, cth;
                if (real) shadow_geometry(w, j, gs, v, dist2, cth);
                dist = real ? sqrtf(dist2) : 0.f;
                if (real && cth > 0.f) {
                    const float3 p = xyz(w.shits.p[j]);
                    const float4 N = w.shits.n[j];
                    ++shadow;
                    dir = v * (1.0f / dist);
                    ray = make_any_ray(p, dir, sc.tmin, dist, __float_as_int(N.w));
                    f = cth * inv_pi / dist2;
                    traced = true;
                }
            }
            const float tlo = ray.tmin * (1.0f - AMBIG_T), tnear = ray.tmin * (1.0f + AMBIG_T);
            bool fin = !traced;  // the lane has its answer
            unsigned todo = __ballot_sync(FULL, traced);
            while (todo) {
                // the lanes of one job walk that job's BVH
                const int leader = __ffs(todo) - 1;
                const int jl = __shfl_sync(FULL, job, leader);
                const unsigned grp = __ballot_sync(FULL, traced && job == jl) & todo;
                todo &= ~grp;
                const SceneView sc = BATCH ? w.jobs[jl].sc : w.job0.sc;  // in registers for the walk
                // direction signs of the leader's ray (the packet's rays are nearly parallel)
                const unsigned dsign = __shfl_sync(
                    FULL, (dir.x < 0.f ? 1u : 0u) | (dir.y < 0.f ? 2u : 0u) | (dir.z < 0.f ? 4u : 0u), leader);
                auto leaf = [&](int tri) {  // the lane's any-hit test of one triangle
                    if (COUNT) ts.tris++;
                    if ((unsigned)tri >= (unsigned)sc.num_tris) {
                        raise_error(w.status, RP_ERR_INVALID_ARG);
                        fin = true;
                        return;
                    }
                    if (tri == ray.exclude) return;
                    float t, margin;
                    uint32_t orig;
                    const bool inside = tri_intersect(sc.tris, tri, ray.o, dir, t, orig, margin);
                    if (EXACT && t > tlo && t < ray.tmax * (1.0f + AMBIG_T) &&
                        (fabsf(margin) < AMBIG_BARY || (inside && t < tnear)))
                        st.amb_t = fminf(st.amb_t, t);
                    if (!inside || !(t > ray.tmin) || !(t < ray.tmax)) return;
                    st.blocked = true;
                    if (!EXACT || (fabsf(margin) >= AMBIG_BARY && t >= tnear)) {
                        st.clear = true;
                        fin = true;
                        blk_leaf = tri;
                    }
                };
                if (sc.num_nodes == 0) {
                    if (((grp >> lane) & 1u) && sc.num_tris > 0) leaf(0);
                    continue;
                }
                const int iter_cap = sc.iter_cap;
                int iters = 0;
                // the packet's items are neighbouring tiles towards one source (two at the edge
                // of a group): it starts where the warp's last packet towards the leader's source
                // found a blocker, else in that source's region (any start gives the same answers)
                const int pk_gs = __shfl_sync(FULL, my_gs, leader);
                int start_node = (hint > 0 && pk_gs == hint_gs) ? hint : __shfl_sync(FULL, start, leader);
                if (w.src_hint && first && !(hint > 0 && pk_gs == hint_gs)) {
                    // another warp's latest hint towards this source (the previous group of tiles)
                    int th = 0;
                    if (lane == leader) th = __ldcg(w.src_hint + (size_t)pk_gs * SRC_HINT_STRIDE);
                    th = __shfl_sync(FULL, th, leader);
                    if (th > 0 && th < sc.num_nodes) start_node = th;
                }
                // walks from start_node, then from SHADOW_HINT_UP levels further up (escalate
                // times, at most twice: the walks of one packet then visit a well-formed tree's
                // nodes at most four times, within the iteration cap), then from the root, each
                // for the lanes still without an answer
                const int esc = min(w.escalate, 2);
                int from = start_node;
                for (int phase = 0; phase <= esc + 1; ++phase) {
                    if (phase > 0) {
                        if (from == 0) break;  // the root's walk answered every lane
                        from = (phase <= esc && sc.up && (unsigned)from < (unsigned)sc.num_nodes) ? sc.up[from] : 0;
                    }
                    int node = from, sp = 0;
                    // lanes of the group that reach `node` and have no answer yet
                    unsigned mask = grp & ~__ballot_sync(FULL, fin);
                    if (!mask) break;
                    if (COUNT && lane == 0) ts.walks++;
                    while (mask) {
                        if (++iters > iter_cap) {
                            if (lane == 0) raise_error(w.status, RP_ERR_TIMEOUT);
                            break;
                        }
                        if ((unsigned)node >= (unsigned)sc.num_nodes) {
                            if (lane == 0) raise_error(w.status, RP_ERR_INVALID_ARG);
                            break;
                        }
                        const bool need = (mask >> lane) & 1u;
                        if (COUNT && need) ts.nodes++;
                        if (COUNT && lane == 0) ts.steps++;
                        const float4 *np = sc.nodes + 4 * node;
                        const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
                        const float a0 = n0.x * ray.idir.x - ray.ood.x, b0 = n0.y * ray.idir.x - ray.ood.x;
                        const float a1 = n0.z * ray.idir.y - ray.ood.y, b1 = n0.w * ray.idir.y - ray.ood.y;
                        const float a2 = n2.x * ray.idir.z - ray.ood.z, b2 = n2.y * ray.idir.z - ray.ood.z;
                        const float c0min = slab_in(a0, b0, a1, b1, a2, b2, ray.tmin);
                        const float c0max = slab_out(a0, b0, a1, b1, a2, b2, ray.tmax);
                        const float a3 = n1.x * ray.idir.x - ray.ood.x, b3 = n1.y * ray.idir.x - ray.ood.x;
                        const float a4 = n1.z * ray.idir.y - ray.ood.y, b4 = n1.w * ray.idir.y - ray.ood.y;
                        const float a5 = n2.z * ray.idir.z - ray.ood.z, b5 = n2.w * ray.idir.z - ray.ood.z;
                        const float c1min = slab_in(a3, b3, a4, b4, a5, b5, ray.tmin);
                        const float c1max = slab_out(a3, b3, a4, b4, a5, b5, ray.tmax);
                        const bool h0 = need && c0min <= c0max, h1 = need && c1min <= c1max;
                        const int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
                        if (h0 && ch0 < 0) leaf(~ch0);
                        if (h1 && ch1 < 0 && !fin) leaf(~ch1);
                        const unsigned m0 = __ballot_sync(FULL, h0 && ch0 >= 0 && !fin);
                        const unsigned m1 = __ballot_sync(FULL, h1 && ch1 >= 0 && !fin);
                        if (m0 && m1) {
                            // the child on the side the rays head to goes first: on the node's
                            // split axis, the higher child for rays heading up the axis
                            const int split = __float_as_int(n3.z);
                            const bool swap = (((dsign >> (split & 3)) ^ (unsigned)(split >> 2)) & 1u) == 0u;
                            if (sp >= STACK_DEPTH) {
                                if (lane == 0) raise_error(w.status, RP_ERR_STACK_OVERFLOW);
                                break;
                            }
                            if (lane == 0) {
                                sn[sp] = swap ? ch0 : ch1;
                                sm[sp] = swap ? m0 : m1;
                            }
                            __syncwarp();
                            ++sp;
                            node = swap ? ch1 : ch0;
                            mask = swap ? m1 : m0;
                        } else if (m0) {
                            node = ch0;
                            mask = m0;
                        } else if (m1) {
                            node = ch1;
                            mask = m1;
                        } else {
                            // pop until an entry still has lanes without an answer
                            const unsigned answered = __ballot_sync(FULL, fin);
                            mask = 0;
                            while (mask == 0 && sp > 0) {
                                --sp;
                                node = sn[sp];
                                mask = sm[sp] & ~answered;
                            }
                        }
                    }
                    __syncwarp();
                }
                // the next hint: SHADOW_HINT_UP levels above the first blocking leaf of this group
                const unsigned cl = __ballot_sync(FULL, ((grp >> lane) & 1u) && st.clear);
                if (cl && sc.anc) {
                    const int src_lane = __ffs(cl) - 1;
                    int a = 0;
                    if (lane == src_lane && (unsigned)blk_leaf < (unsigned)sc.num_tris) {
                        a = sc.anc[blk_leaf];
                        if ((unsigned)a >= (unsigned)sc.num_nodes) a = 0;
                    }
                    a = __shfl_sync(FULL, a, src_lane);
                    if (a > 0) {
                        hint = a;
                        hint_gs = pk_gs;
                    }
                }
            }
            first = false;
            if (!traced) continue;
            const bool amb = EXACT && !st.clear && st.amb_t < INFINITY;
            if (amb) {
                const unsigned long long r = warp_append(&w.ctr->n_rerun);
                if (r < w.rerun_cap) {
                    w.rerun[r] = item;
                    continue;
                }
            }
            if (!st.blocked) {
                unsigned long long j;
                int gs;
                item_slot(w, BATCH, job, item, j, gs);
                ++contrib;
                shadow_contribution(w, acc, j, gs, f, dist);
            }
        }
        // the block's last hint, for the warp that takes the next group of tiles
        if (w.src_hint && hint > 0 && hint_gs >= 0 && lane == 0) __stcg(w.src_hint + (size_t)hint_gs * SRC_HINT_STRIDE, hint);
    }
    acc_counters(acc, 0.0, 0.0, 0ull, 0ull, 0ull, shadow, contrib, 0ull, ts);
    acc_flush(acc, w.stats, w.k.B, 1);
}

// FP64 decisions for the shadow rays whose FP32 visibility was rounding-sensitive
__global__ void __launch_bounds__(SHADOW_THREADS) k_shadow_exact(TraceWork w, unsigned long long chunk)
{
    const unsigned long long n = min(w.ctr->n_rerun, w.rerun_cap);
    if (n == 0) return;  // nothing queued (the whole grid)
    __shared__ int sstack[SMEM_STACK * SHADOW_THREADS];
    __shared__ BlockAcc acc;
    acc_init(acc);
    __syncthreads();
    unsigned long long contrib = 0;
    (void)chunk;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        int job, gs;
        unsigned long long j;
        item_target(w, w.njobs > 1, w.rerun[i], job, j, gs);
        const SceneView &sc = w.njobs > 1 ? w.jobs[job].sc : w.job0.sc;
        const float4 P = w.shits.p[j], N = w.shits.n[j], lo = w.hits.plo[w.horder.perm[j]];
        const float4 cs = __ldg(w.pos + gs);
        const D3 pd = {(double)P.x + lo.x, (double)P.y + lo.y, (double)P.z + lo.z};
        const double vx = (double)cs.x - pd.x, vy = (double)cs.y - pd.y, vz = (double)cs.z - pd.z;
        const double dd = sqrt(vx * vx + vy * vy + vz * vz);
        double te;
        const int blk = traverse_exact<true>(sc, pd, D3{vx / dd, vy / dd, vz / dd}, sc.tmin_d, dd,
                                             __float_as_int(N.w), sstack + threadIdx.x, te, w.status);
        if (blk < 0) {
            const float3 v = xyz(cs) - xyz(P);
            const float dist2 = dot(v, v), dist = sqrtf(dist2);
            const float cth = dot(xyz(N), v) / dist;
            ++contrib;
            shadow_contribution(w, acc, j, gs, cth * (1.0f / PI_F) / dist2, dist);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd((unsigned long long *)&w.stats->fp64_reruns, n);
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(FULL, contrib, o);
    if ((threadIdx.x & 31) == 0 && contrib) atomicAdd(&acc.contrib, contrib);
    acc_flush(acc, w.stats, w.k.B, 1);
}

// Direct sound of the group's sources: distance, time and bin in FP64, the
// visibility ray in FP32 (re-decided in FP64 when rounding-sensitive).
// Start node of each source's shadow-ray packets: from the root, into the child whose
// box alone holds the source, while that child's box is at least region_frac of the
// scene's largest extent.  Rays that end at the source cross this region last; the
// packets walk it first, then (the lanes still without an answer) the whole tree.
__global__ void k_src_region(TraceWork w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.k.S) return;
    const int gs = w.src_base + i;
    const SceneJob &J = w.njobs > 1 ? w.jobs[w.src_job[gs]] : w.job0;
    const SceneView &sc = J.sc;
    const float4 s4 = __ldg(w.pos + gs);
    const float lim = w.region_frac * fmaxf(sc.ext[0], fmaxf(sc.ext[1], sc.ext[2]));
    int node = 0;
    for (int d = 0; d < STACK_DEPTH && sc.num_nodes > 0 && w.region_frac > 0.f; ++d) {
        if ((unsigned)node >= (unsigned)sc.num_nodes) {
            node = 0;
            break;
        }
        const float4 *np = sc.nodes + 4 * node;
        const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
        const bool in0 = s4.x >= n0.x && s4.x <= n0.y && s4.y >= n0.z && s4.y <= n0.w && s4.z >= n2.x && s4.z <= n2.y;
        const bool in1 = s4.x >= n1.x && s4.x <= n1.y && s4.y >= n1.z && s4.y <= n1.w && s4.z >= n2.z && s4.z <= n2.w;
        const int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
        const float e0 = fmaxf(n0.y - n0.x, fmaxf(n0.w - n0.z, n2.y - n2.x));
        const float e1 = fmaxf(n1.y - n1.x, fmaxf(n1.w - n1.z, n2.w - n2.z));
        // the child whose box alone holds the source
        const bool take0 = in0 && !in1 && ch0 >= 0;
        const bool take1 = in1 && !in0 && ch1 >= 0;
        if (!take0 && !take1) break;
        const float ext = take0 ? e0 : e1;
        if (ext < lim) break;
        node = take0 ? ch0 : ch1;
    }
    w.src_node[gs] = node;
    if (w.src_hint) w.src_hint[(size_t)gs * SRC_HINT_STRIDE] = 0;
}

__global__ void __launch_bounds__(128) k_direct(TraceWork w)
{
    __shared__ int sstack[SMEM_STACK * 128];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.k.S) return;
    const int gs = w.src_base + i;
    const int job = w.njobs > 1 ? w.src_job[gs] : 0;
    const SceneJob &J = w.njobs > 1 ? w.jobs[job] : w.job0;
    const float4 l4 = __ldg(w.pos + J.lis), s4 = __ldg(w.pos + gs);
    const double vx = (double)s4.x - l4.x, vy = (double)s4.y - l4.y, vz = (double)s4.z - l4.z;
    const double dist = sqrt(vx * vx + vy * vy + vz * vz);
    const float3 dir = mk3((float)(vx / dist), (float)(vy / dist), (float)(vz / dist));
    TravStats ts = {0u, 0u};
    float tt;
    bool amb = false;
    int blk = traverse<true, false, true>(J.sc, xyz(l4), dir, J.sc.tmin, (float)dist, -1, sstack + threadIdx.x, tt,
                                          ts, w.status, &amb);
    if (amb) {
        double te;
        blk = traverse_exact<true>(J.sc, D3{(double)l4.x, (double)l4.y, (double)l4.z},
                                   D3{vx / dist, vy / dist, vz / dist}, J.sc.tmin_d, dist, -1, sstack + threadIdx.x,
                                   te, w.status);
    }
    rp_direct out;
    out.visible = blk < 0 ? 1 : 0;
    out.dist = (float)dist;
    const double time = dist / (double)w.k.c;
    out.time = (float)time;
    out.energy = blk < 0 ? (float)(1.0 / (4.0 * 3.14159265358979323846 * dist * dist)) : 0.0f;
    const double binf = floor(time * (double)w.k.rate);
    out.bin = binf < 2147483520.0 ? (int)binf : 0x7fffffff;
    float Y[MAXK];
    sh_eval(w.k.sh_order, dir.x, dir.y, dir.z, Y);
    for (int kk = 0; kk < MAXK; ++kk) out.sh[kk] = kk < w.k.K ? out.energy * Y[kk] : 0.f;
    w.direct[gs] = out;
}

}  // namespace

void launch_setup(const TraceWork &w, int wave, cudaStream_t st)
{
    k_setup<<<wave == 0 ? (w.njobs + 127) / 128 : 1, 128, 0, st>>>(w, wave);
}

void launch_item_prefix(const TraceWork &w, cudaStream_t st) { k_item_prefix<<<1, 32, 0, st>>>(w); }

void launch_plan_block(const TraceWork &w, unsigned long long begin, unsigned long long count, cudaStream_t st)
{
    k_plan_block<<<1, 32, 0, st>>>(w, begin, count);
}

void launch_refill_plan(const TraceWork &w, unsigned long long candidates, cudaStream_t st)
{
    k_refill_plan<<<1, REFILL_THREADS, 0, st>>>(w, candidates);
}

void launch_plan_apply(const TraceWork &w, cudaStream_t st) { k_plan_apply<<<1, 32, 0, st>>>(w); }

void launch_spec_fold(const TraceWork &w, unsigned long long count, cudaStream_t st)
{
    const int blocks = (int)std::max(1ull, std::min<unsigned long long>((count + 255) / 256, 4096ull));
    k_spec_fold<<<blocks, 256, 0, st>>>(w, count);
}

void launch_hit_order(const TraceWork &w, int blocks, cudaStream_t st)
{
    cudaMemsetAsync(w.horder.cnt, 0, sizeof(uint32_t) * ((size_t)w.horder.ncells + 1), st);
    k_hit_cells<<<blocks, 256, 0, st>>>(w);
    launch_scan_u32(w.horder.cnt, w.horder.cnt, w.horder.ncells, w.scan_part, st);
    k_hit_scatter<<<blocks, 256, 0, st>>>(w);
    if (w.rid_end) k_hits_kept<<<1, 32, 0, st>>>(w);
    k_hit_gather<<<blocks, 256, 0, st>>>(w);
}

template <typename R, bool BATCH>
void launch_paths_r(const TraceWork &w, int blocks, cudaStream_t st)
{
    const bool hash = (w.k.flags & RP_FLAG_RAY_HASH) && w.ray_hash;
    const bool count = (w.k.flags & RP_FLAG_COUNT_VISITS) != 0;
    if (hash && count) k_paths<R, true, true, BATCH><<<blocks, PATH_THREADS, 0, st>>>(w);
    else if (hash) k_paths<R, true, false, BATCH><<<blocks, PATH_THREADS, 0, st>>>(w);
    else if (count) k_paths<R, false, true, BATCH><<<blocks, PATH_THREADS, 0, st>>>(w);
    else k_paths<R, false, false, BATCH><<<blocks, PATH_THREADS, 0, st>>>(w);
}

void launch_paths(const TraceWork &w, int blocks, cudaStream_t st)
{
    if (w.plan == 2) {  // a store pass (one job, FP64 paths, no hashes or visit counts)
        k_paths<double, false, false, false, true><<<blocks, PATH_THREADS, 0, st>>>(w);
        return;
    }
    const bool batch = !w.wave_mode;
    if (w.k.flags & RP_FLAG_FP32_PATHS) {
        if (batch) launch_paths_r<float, true>(w, blocks, st);
        else launch_paths_r<float, false>(w, blocks, st);
    } else {
        if (batch) launch_paths_r<double, true>(w, blocks, st);
        else launch_paths_r<double, false>(w, blocks, st);
    }
}

template <bool BATCH>
void launch_shadow_b(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st)
{
    const bool count = (w.k.flags & RP_FLAG_COUNT_VISITS) != 0;
    const bool exact = (w.k.flags & RP_FLAG_FP32_PATHS) == 0;
    if (w.shadow_packets) {
        if (count && exact) k_shadow_packet<true, true, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
        else if (count) k_shadow_packet<true, false, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
        else if (exact) k_shadow_packet<false, true, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
        else k_shadow_packet<false, false, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
        return;
    }
    if (count && exact) k_shadow<true, true, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
    else if (count) k_shadow<true, false, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
    else if (exact) k_shadow<false, true, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
    else k_shadow<false, false, BATCH><<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
}

void launch_shadow(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st)
{
    if (w.njobs > 1) launch_shadow_b<true>(w, chunk, blocks, st);
    else launch_shadow_b<false>(w, chunk, blocks, st);
}

void launch_shadow_exact(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st)
{
    if ((w.k.flags & RP_FLAG_FP32_PATHS) == 0) k_shadow_exact<<<blocks, SHADOW_THREADS, 0, st>>>(w, chunk);
}

void launch_src_region(const TraceWork &w, cudaStream_t st)
{
    if (w.k.S > 0 && w.src_node) k_src_region<<<(w.k.S + 127) / 128, 128, 0, st>>>(w);
}

void launch_direct(const TraceWork &w, cudaStream_t st)
{
    if (w.k.S > 0 && w.direct) k_direct<<<(w.k.S + 127) / 128, 128, 0, st>>>(w);
}

int paths_occupancy(int flags)
{
    int n = 0;
    if (flags & RP_FLAG_FP32_PATHS)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_paths<float, false, false, false>, PATH_THREADS, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_paths<double, false, false, false>, PATH_THREADS, 0);
    return n > 0 ? n : 1;
}

int shadow_occupancy(int flags)
{
    // the persistent grid must fit both shadow-ray kernels
    int n = 0, m = 0;
    if (flags & RP_FLAG_FP32_PATHS) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shadow<false, false, false>, SHADOW_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_shadow_packet<false, false, false>, SHADOW_THREADS, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_shadow<false, true, false>, SHADOW_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_shadow_packet<false, true, false>, SHADOW_THREADS, 0);
    }
    n = std::min(n, m);
    return n > 0 ? n : 1;
}

}  // namespace rp
