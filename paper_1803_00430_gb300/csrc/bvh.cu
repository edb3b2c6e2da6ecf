// bvh.cu -- device construction of the scene's bounding-volume hierarchy.
//
// The paper's ray tracer leaves its acceleration structure unspecified (Section 6
// "Performance" only states that cost grows logarithmically with scene size).  This
// file builds the BVH entirely on the GPU:
//   1. per-triangle bounds and centroids, checked for non-finite values;
//   2. 30-bit Morton codes of the centroids;
//   3. a stable LSD radix sort (8-bit digits) of (code, triangle) pairs;
//   4. the hierarchy by parallel locally-ordered clustering (PLOC, Meister & Bittner,
//      IEEE TVCG 2018): in Morton order, every cluster finds the neighbour within
//      +-PLOC_RADIUS positions whose union box has the smallest surface area;
//      mutual nearest pairs merge into a new node; the survivors are compacted, and
//      rounds repeat until one cluster is left.  Node ids come from prefix sums
//      (the root is node 0), so the build is deterministic;
//   5. packing into 64-byte nodes holding both children's boxes, and 48-byte
//      triangles in leaf order; per-material constants.
#include <cstdio>
#include <vector>

#include "internal.cuh"

namespace rp {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__device__ __forceinline__ bool finite3(float3 v) { return isfinite(v.x) && isfinite(v.y) && isfinite(v.z); }

// --- 1. triangle bounds ------------------------------------------------------
__global__ void k_tri_prep(const float *__restrict__ verts, const int32_t *__restrict__ tris,
                           const int32_t *__restrict__ tmat, int nv, int nt, int nmat,
                           float4 *__restrict__ blo, float4 *__restrict__ bhi,
                           float *__restrict__ partial, int *status)
{
    // partial[blockIdx * 12]: centroid lo/hi (6), vertex lo/hi (6)
    __shared__ float red[12][256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float cl[3] = {INFINITY, INFINITY, INFINITY}, ch[3] = {-INFINITY, -INFINITY, -INFINITY};
    float vl[3] = {INFINITY, INFINITY, INFINITY}, vh[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < nt) {
        const int a = tris[3 * i], b = tris[3 * i + 1], c = tris[3 * i + 2];
        const int m = tmat[i];
        if (a < 0 || a >= nv || b < 0 || b >= nv || c < 0 || c >= nv || m < 0 || m >= nmat) {
            raise_error(status, RP_ERR_INVALID_ARG);
        } else {
            const float3 p0 = mk3(verts[3 * a], verts[3 * a + 1], verts[3 * a + 2]);
            const float3 p1 = mk3(verts[3 * b], verts[3 * b + 1], verts[3 * b + 2]);
            const float3 p2 = mk3(verts[3 * c], verts[3 * c + 1], verts[3 * c + 2]);
            if (!finite3(p0) || !finite3(p1) || !finite3(p2)) {
                raise_error(status, RP_ERR_NAN_INPUT);
            } else {
                const float3 lo = mk3(fminf(p0.x, fminf(p1.x, p2.x)), fminf(p0.y, fminf(p1.y, p2.y)),
                                      fminf(p0.z, fminf(p1.z, p2.z)));
                const float3 hi = mk3(fmaxf(p0.x, fmaxf(p1.x, p2.x)), fmaxf(p0.y, fmaxf(p1.y, p2.y)),
                                      fmaxf(p0.z, fmaxf(p1.z, p2.z)));
                blo[i] = make_float4(lo.x, lo.y, lo.z, 0.f);
                bhi[i] = make_float4(hi.x, hi.y, hi.z, 0.f);
                const float3 cc = mk3((p0.x + p1.x + p2.x) * (1.f / 3.f), (p0.y + p1.y + p2.y) * (1.f / 3.f),
                                      (p0.z + p1.z + p2.z) * (1.f / 3.f));
                cl[0] = ch[0] = cc.x;
                cl[1] = ch[1] = cc.y;
                cl[2] = ch[2] = cc.z;
                vl[0] = lo.x; vl[1] = lo.y; vl[2] = lo.z;
                vh[0] = hi.x; vh[1] = hi.y; vh[2] = hi.z;
            }
        }
    }
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = cl[a];
        red[3 + a][threadIdx.x] = ch[a];
        red[6 + a][threadIdx.x] = vl[a];
        red[9 + a][threadIdx.x] = vh[a];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int a = 0; a < 3; ++a) {
                red[a][threadIdx.x] = fminf(red[a][threadIdx.x], red[a][threadIdx.x + s]);
                red[3 + a][threadIdx.x] = fmaxf(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + s]);
                red[6 + a][threadIdx.x] = fminf(red[6 + a][threadIdx.x], red[6 + a][threadIdx.x + s]);
                red[9 + a][threadIdx.x] = fmaxf(red[9 + a][threadIdx.x], red[9 + a][threadIdx.x + s]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 12) partial[blockIdx.x * 12 + threadIdx.x] = red[threadIdx.x][0];
}

// bounds[0..11] = centroid lo/hi, vertex lo/hi
__global__ void k_reduce_bounds(const float *__restrict__ partial, int nblk, float *__restrict__ bounds)
{
    const int a = threadIdx.x;  // 12 threads
    if (a >= 12) return;
    const bool is_min = (a % 6) < 3;
    float v = is_min ? INFINITY : -INFINITY;
    for (int b = 0; b < nblk; ++b) v = is_min ? fminf(v, partial[b * 12 + a]) : fmaxf(v, partial[b * 12 + a]);
    bounds[a] = v;
}

// --- 2. Morton codes -----------------------------------------------------------
__device__ __forceinline__ uint32_t expand_bits(uint32_t v)
{
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__global__ void k_morton(const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                         const float *__restrict__ bounds, int nt, uint32_t *__restrict__ keys,
                         uint32_t *__restrict__ vals)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const float4 lo = blo[i], hi = bhi[i];
    float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        const float ext = bounds[3 + a] - bounds[a];
        float u = ext > 0.f ? (c[a] - bounds[a]) / ext : 0.5f;
        u = fminf(fmaxf(u, 0.f), 1.f);
        q[a] = min((uint32_t)(u * 1024.f), 1023u);
    }
    keys[i] = (expand_bits(q[0]) << 2) | (expand_bits(q[1]) << 1) | expand_bits(q[2]);
    vals[i] = (uint32_t)i;
}

// --- 3. stable LSD radix sort, 8-bit digits ---------------------------------------
__global__ void k_rs_hist(const uint32_t *__restrict__ keys, int n, int shift, int nblk,
                          uint32_t *__restrict__ hist)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; ++it) {
        const int idx = base + it * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of n uint32 in place, one block of 1024 threads
__global__ void k_scan_u32(uint32_t *__restrict__ a, int n, uint32_t *__restrict__ total)
{
    __shared__ uint32_t warp_sums[32];
    const int t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int b = t * per, e = min(n, b + per);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += a[i];
    // block exclusive scan of s
    const int lane = t & 31, wid = t >> 5;
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - s + (wid > 0 ? warp_sums[wid - 1] : 0u);
    for (int i = b; i < e; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
    if (total && t == 1023) *total = run;
}

__global__ void k_rs_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int n, int shift,
                             int nblk, const uint32_t *__restrict__ hist)
{
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    run[t] = hist[t * nblk + blockIdx.x];
    for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][t] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; ++it) {
        const int idx = base + it * RS_THREADS + t;
        const bool valid = idx < n;
        const uint32_t k = valid ? kin[idx] : 0u;
        const uint32_t v = valid ? vin[idx] : 0u;
        const uint32_t d = (k >> shift) & 255u;
        const unsigned peers = __match_any_sync(FULL, valid ? d : 0x10000u + (uint32_t)lane);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t o = run[d];
            for (int w = 0; w < wid; ++w) o += wcnt[w][d];
            kout[o + rank] = k;
            vout[o + rank] = v;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < RS_THREADS / 32; ++w) {
            add += wcnt[w][t];
            wcnt[w][t] = 0;
        }
        run[t] += add;
        __syncthreads();
    }
}

// --- 4. PLOC hierarchy -------------------------------------------------------------
constexpr int PLOC_RADIUS = 32;

__device__ __forceinline__ float union_area(float4 al, float4 ah, float4 bl, float4 bh)
{
    const float dx = fmaxf(ah.x, bh.x) - fminf(al.x, bl.x);
    const float dy = fmaxf(ah.y, bh.y) - fminf(al.y, bl.y);
    const float dz = fmaxf(ah.z, bh.z) - fminf(al.z, bl.z);
    return dx * dy + dy * dz + dz * dx;  // half the surface area
}

// leaves in Morton order as the first clusters
__global__ void k_ploc_init(int n, const uint32_t *__restrict__ order, const float4 *__restrict__ blo,
                            const float4 *__restrict__ bhi, int *__restrict__ cref, float4 *__restrict__ clo,
                            float4 *__restrict__ chi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = order[i];
    cref[i] = ~i;
    clo[i] = blo[t];
    chi[i] = bhi[t];
}

// nearest neighbour of every cluster within the window; the pair key (area, lower
// index, higher index) is compared lexicographically, so the smallest pair overall
// is always mutual and every round merges at least once
__global__ void k_ploc_nn(int c, const float4 *__restrict__ clo, const float4 *__restrict__ chi,
                          int *__restrict__ nn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c) return;
    const float4 li = clo[i], hi = chi[i];
    float best = INFINITY;
    int bj = -1, blo_ = 0, bhi_ = 0;
    const int j0 = max(0, i - PLOC_RADIUS), j1 = min(c - 1, i + PLOC_RADIUS);
    for (int j = j0; j <= j1; ++j) {
        if (j == i) continue;
        const float a = union_area(li, hi, clo[j], chi[j]);
        const int lo = min(i, j), hh = max(i, j);
        if (a < best || (a == best && (lo < blo_ || (lo == blo_ && hh < bhi_)))) {
            best = a;
            bj = j;
            blo_ = lo;
            bhi_ = hh;
        }
    }
    nn[i] = bj;
}

// keep[i]: cluster i survives the round (alone, or as the merged pair's lower index);
// merge[i]: it is the lower index of a mutual pair
__global__ void k_ploc_flags(int c, const int *__restrict__ nn, uint32_t *__restrict__ keep,
                             uint32_t *__restrict__ merge)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c) return;
    const int j = nn[i];
    const bool mutual = j >= 0 && nn[j] == i;
    merge[i] = mutual && i < j ? 1u : 0u;
    keep[i] = mutual && i > j ? 0u : 1u;
}

// merges (new node id = c - 2 - rank among this iteration's merges) and compaction
__global__ void k_ploc_merge(int c, const int *__restrict__ cref, const float4 *__restrict__ clo,
                             const float4 *__restrict__ chi, const int *__restrict__ nn,
                             const uint32_t *__restrict__ keep, const uint32_t *__restrict__ kpos,
                             const uint32_t *__restrict__ merge, const uint32_t *__restrict__ mpos,
                             int2 *__restrict__ child, float4 *__restrict__ nlo, float4 *__restrict__ nhi,
                             int *__restrict__ parent_int, int *__restrict__ parent_leaf, int *__restrict__ oref,
                             float4 *__restrict__ olo, float4 *__restrict__ ohi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c || !keep[i]) return;
    const uint32_t pos = kpos[i];
    if (merge[i]) {
        const int j = nn[i];
        const int id = c - 2 - (int)mpos[i];
        const int a = cref[i], b = cref[j];
        const float4 al = clo[i], ah = chi[i], bl = clo[j], bh = chi[j];
        const float4 lo = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f);
        const float4 hi = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f);
        child[id] = make_int2(a, b);
        nlo[id] = lo;
        nhi[id] = hi;
        if (a < 0) parent_leaf[~a] = id;
        else parent_int[a] = id;
        if (b < 0) parent_leaf[~b] = id;
        else parent_int[b] = id;
        oref[pos] = id;
        olo[pos] = lo;
        ohi[pos] = hi;
    } else {
        oref[pos] = cref[i];
        olo[pos] = clo[i];
        ohi[pos] = chi[i];
    }
}

__device__ __forceinline__ void child_box(int c, const uint32_t *__restrict__ order,
                                          const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                                          const float4 *nlo, const float4 *nhi, float4 &lo, float4 &hi)
{
    if (c < 0) {
        const uint32_t t = order[~c];
        lo = blo[t];
        hi = bhi[t];
    } else {
        lo = nlo[c];
        hi = nhi[c];
    }
}

// the node SHADOW_HINT_UP levels above each leaf (the root where the tree is shallower)
__global__ void k_leaf_anc(int n, const int *__restrict__ parent_int, const int *__restrict__ parent_leaf,
                           int *__restrict__ anc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = parent_leaf[i];
    for (int u = 1; u < SHADOW_HINT_UP && p > 0; ++u) p = parent_int[p];
    anc[i] = p > 0 ? p : 0;
}

// the node SHADOW_HINT_UP levels above each internal node (the root above the top levels)
__global__ void k_node_up(int n, const int *__restrict__ parent_int, int *__restrict__ up)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = i;
    for (int u = 0; u < SHADOW_HINT_UP && p > 0; ++u) p = parent_int[p];
    up[i] = p > 0 ? p : 0;
}

__global__ void k_depth(int n, const int *__restrict__ parent_int, const int *__restrict__ parent_leaf,
                        int *__restrict__ max_depth)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = parent_leaf[i], d = 1;
    while (p > 0 && d < 4096) {
        p = parent_int[p];
        ++d;
    }
    atomicMax(max_depth, d);
}

// --- 6. packing ----------------------------------------------------------------------
__global__ void k_pack_nodes(int n, const uint32_t *__restrict__ order, const float4 *__restrict__ blo,
                             const float4 *__restrict__ bhi, const int2 *__restrict__ child,
                             const float4 *__restrict__ nlo, const float4 *__restrict__ nhi, float pad,
                             float4 *__restrict__ nodes)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int2 c = child[i];
    float4 l0, h0, l1, h1;
    child_box(c.x, order, blo, bhi, nlo, nhi, l0, h0);
    child_box(c.y, order, blo, bhi, nlo, nhi, l1, h1);
    // conservative padding: the slab and triangle tests round differently
    nodes[4 * i + 0] = make_float4(l0.x - pad, h0.x + pad, l0.y - pad, h0.y + pad);
    nodes[4 * i + 1] = make_float4(l1.x - pad, h1.x + pad, l1.y - pad, h1.y + pad);
    nodes[4 * i + 2] = make_float4(l0.z - pad, h0.z + pad, l1.z - pad, h1.z + pad);
    // split code: the axis along which the children's centres lie farthest apart (bits
    // 0-1) and whether the first child's centre is the higher one on it (bit 2); a
    // packet of shadow rays walks first the child on the side its rays come from
    const float d[3] = {(l1.x + h1.x) - (l0.x + h0.x), (l1.y + h1.y) - (l0.y + h0.y),
                        (l1.z + h1.z) - (l0.z + h0.z)};
    const float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    const int axis = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    const int split = axis | (d[axis] < 0.f ? 4 : 0);
    nodes[4 * i + 3] = make_float4(__int_as_float(c.x), __int_as_float(c.y), __int_as_float(split), 0.f);
}

__global__ void k_pack_tris(int nt, const uint32_t *__restrict__ order, const float *__restrict__ verts,
                            const int32_t *__restrict__ tris, const int32_t *__restrict__ tmat,
                            float4 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int t = (int)order[i];
    if (t < 0 || t >= nt) return;
    const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    const float3 p0 = mk3(verts[3 * a], verts[3 * a + 1], verts[3 * a + 2]);
    const float3 p1 = mk3(verts[3 * b], verts[3 * b + 1], verts[3 * b + 2]);
    const float3 p2 = mk3(verts[3 * c], verts[3 * c + 1], verts[3 * c + 2]);
    out[3 * i + 0] = make_float4(p0.x, p0.y, p0.z, __int_as_float(tmat[t]));
    out[3 * i + 1] = make_float4(p1.x, p1.y, p1.z, __int_as_float(t));
    out[3 * i + 2] = make_float4(p2.x, p2.y, p2.z, 0.f);
}

// per-material constants; the diffuse threshold is computed in double exactly as
// ceil(mean(s_b) * 2^24) so that the diffuse/specular decision is bit-reproducible
__global__ void k_materials(const float *__restrict__ alpha, const float *__restrict__ scat, int nmat, int B,
                            float *__restrict__ a_out, float *__restrict__ s_out, float *__restrict__ wdiff,
                            float *__restrict__ wspec, uint32_t *__restrict__ thr, int *status)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmat) return;
    double sum = 0.0;
    bool bad = false;
    for (int b = 0; b < B; ++b) {
        const float a = alpha[m * B + b], s = scat[m * B + b];
        if (!isfinite(a) || !isfinite(s)) bad = true;
        if (!(a >= 0.f && a <= 1.f && s >= 0.f && s <= 1.f)) bad = true;
        sum += (double)s;
    }
    if (bad) {
        raise_error(status, isfinite(sum) ? RP_ERR_INVALID_ARG : RP_ERR_NAN_INPUT);
        return;
    }
    const double sbar = sum / (double)B;
    thr[m] = (uint32_t)ceil(sbar * 16777216.0);
    for (int b = 0; b < B; ++b) {
        const double s = (double)scat[m * B + b];
        a_out[m * B + b] = alpha[m * B + b];
        s_out[m * B + b] = (float)s;
        wdiff[m * B + b] = sbar > 0.0 ? (float)(s / sbar) : 0.f;
        wspec[m * B + b] = sbar < 1.0 ? (float)((1.0 - s) / (1.0 - sbar)) : 0.f;
    }
}

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
}

}  // namespace

#define RP_TRY(x)                                  \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) { err = e_; goto done; } \
    } while (0)

cudaError_t build_bvh(const BvhBuildArgs &a, BvhOut &out, int *d_status, cudaStream_t st)
{
    cudaError_t err = cudaSuccess;
    const int nt = a.nt;
    const int nblk_tri = (nt + 255) / 256;
    const int nblk_rs = (nt + RS_TILE - 1) / RS_TILE;
    float4 *blo = nullptr, *bhi = nullptr, *nlo = nullptr, *nhi = nullptr;
    float *partial = nullptr, *bounds = nullptr;
    uint32_t *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr, *hist = nullptr;
    int2 *child = nullptr;
    int *pint = nullptr, *pleaf = nullptr, *depth = nullptr, *nn = nullptr, *cref[2] = {nullptr, nullptr};
    float4 *clo[2] = {nullptr, nullptr}, *chi[2] = {nullptr, nullptr};
    uint32_t *keep = nullptr, *kpos = nullptr, *merge = nullptr, *mpos = nullptr;
    float hb[12];
    int hdepth = 0;
    RP_TRY(dalloc(&blo, nt));
    RP_TRY(dalloc(&bhi, nt));
    RP_TRY(dalloc(&partial, (size_t)nblk_tri * 12));
    RP_TRY(dalloc(&bounds, 12));
    RP_TRY(dalloc(&k0, nt));
    RP_TRY(dalloc(&v0, nt));
    RP_TRY(dalloc(&k1, nt));
    RP_TRY(dalloc(&v1, nt));
    RP_TRY(dalloc(&hist, (size_t)256 * nblk_rs));
    RP_TRY(dalloc(&child, nt));
    RP_TRY(dalloc(&pint, nt));
    RP_TRY(dalloc(&pleaf, nt));
    RP_TRY(dalloc(&nn, nt));
    for (int b = 0; b < 2; ++b) {
        RP_TRY(dalloc(&cref[b], nt));
        RP_TRY(dalloc(&clo[b], nt));
        RP_TRY(dalloc(&chi[b], nt));
    }
    RP_TRY(dalloc(&keep, nt + 1));
    RP_TRY(dalloc(&kpos, nt + 1));
    RP_TRY(dalloc(&merge, nt + 1));
    RP_TRY(dalloc(&mpos, nt + 1));
    RP_TRY(dalloc(&nlo, nt));
    RP_TRY(dalloc(&nhi, nt));
    RP_TRY(dalloc(&depth, 1));

    k_tri_prep<<<nblk_tri, 256, 0, st>>>(a.verts, a.tris, a.tri_mat, a.nv, nt, a.nmat, blo, bhi, partial,
                                         d_status);
    k_reduce_bounds<<<1, 32, 0, st>>>(partial, nblk_tri, bounds);
    {
        // invalid indices or non-finite vertices stop the build here
        int hstat = 0;
        RP_TRY(cudaMemcpyAsync(&hstat, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
        RP_TRY(cudaStreamSynchronize(st));
        if (hstat != 0) goto done;
    }
    k_morton<<<nblk_tri, 256, 0, st>>>(blo, bhi, bounds, nt, k0, v0);
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        k_rs_hist<<<nblk_rs, RS_THREADS, 0, st>>>(k0, nt, shift, nblk_rs, hist);
        k_scan_u32<<<1, 1024, 0, st>>>(hist, 256 * nblk_rs, nullptr);
        k_rs_scatter<<<nblk_rs, RS_THREADS, 0, st>>>(k0, v0, k1, v1, nt, shift, nblk_rs, hist);
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    RP_TRY(cudaMemsetAsync(pint, 0xff, sizeof(int) * nt, st));
    RP_TRY(cudaMemsetAsync(pleaf, 0xff, sizeof(int) * nt, st));
    RP_TRY(cudaMemsetAsync(depth, 0, sizeof(int), st));
    if (nt > 1) {
        k_ploc_init<<<nblk_tri, 256, 0, st>>>(nt, v0, blo, bhi, cref[0], clo[0], chi[0]);
        int c = nt, cur = 0;
        for (int round = 0; c > 1; ++round) {
            const int nb = (c + 255) / 256;
            k_ploc_nn<<<nb, 256, 0, st>>>(c, clo[cur], chi[cur], nn);
            k_ploc_flags<<<nb, 256, 0, st>>>(c, nn, keep, merge);
            launch_scan_u32(keep, kpos, c, nullptr, st);
            launch_scan_u32(merge, mpos, c, nullptr, st);
            k_ploc_merge<<<nb, 256, 0, st>>>(c, cref[cur], clo[cur], chi[cur], nn, keep, kpos, merge, mpos, child,
                                             nlo, nhi, pint, pleaf, cref[1 - cur], clo[1 - cur], chi[1 - cur]);
            uint32_t next = 0;
            RP_TRY(cudaMemcpyAsync(&next, kpos + c, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            RP_TRY(cudaStreamSynchronize(st));
            if ((int)next >= c || round > nt) {  // no merge: cannot happen (see k_ploc_nn)
                err = cudaErrorUnknown;
                goto done;
            }
            c = (int)next;
            cur = 1 - cur;
        }
        k_depth<<<nblk_tri, 256, 0, st>>>(nt, pint, pleaf, depth);
    }
    RP_TRY(cudaGetLastError());
    RP_TRY(cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, st));
    RP_TRY(cudaMemcpyAsync(&hdepth, depth, sizeof(int), cudaMemcpyDeviceToHost, st));
    RP_TRY(cudaStreamSynchronize(st));
    {
        float diag2 = 0.f, amax = 0.f;
        for (int k = 0; k < 3; ++k) {
            out.lo[k] = hb[6 + k];
            out.hi[k] = hb[9 + k];
            const float e = hb[9 + k] - hb[6 + k];
            diag2 += e * e;
            amax = fmaxf(amax, fmaxf(fabsf(hb[6 + k]), fabsf(hb[9 + k])));
        }
        const float diag = sqrtf(diag2);
        double dd2 = 0.0;
        for (int k = 0; k < 3; ++k) dd2 += ((double)hb[9 + k] - hb[6 + k]) * ((double)hb[9 + k] - hb[6 + k]);
        out.tmin_d = a.ray_eps > 0.f ? (double)a.ray_eps : 1e-6 * sqrt(dd2);
        out.tmin = a.ray_eps > 0.f ? a.ray_eps : (float)out.tmin_d;
        out.max_depth = nt > 1 ? hdepth : 0;
        const float pad = 1e-6f * (amax + diag) + 1e-30f;
        if (nt > 1)
            k_pack_nodes<<<(nt - 1 + 255) / 256, 256, 0, st>>>(nt, v0, blo, bhi, child, nlo, nhi, pad,
                                                              out.nodes);
        k_pack_tris<<<nblk_tri, 256, 0, st>>>(nt, v0, a.verts, a.tris, a.tri_mat, out.tris);
        if (out.pleaf) RP_TRY(cudaMemcpyAsync(out.pleaf, pleaf, sizeof(int) * nt, cudaMemcpyDeviceToDevice, st));
        if (out.pint && nt > 1)
            RP_TRY(cudaMemcpyAsync(out.pint, pint, sizeof(int) * (nt - 1), cudaMemcpyDeviceToDevice, st));
        if (out.anc) {
            if (nt > 1) k_leaf_anc<<<nblk_tri, 256, 0, st>>>(nt, pint, pleaf, out.anc);
            else RP_TRY(cudaMemsetAsync(out.anc, 0, sizeof(int) * nt, st));
        }
        if (out.up && nt > 1) k_node_up<<<(nt - 1 + 255) / 256, 256, 0, st>>>(nt - 1, pint, out.up);
        k_materials<<<(a.nmat + 127) / 128, 128, 0, st>>>(a.alpha, a.scat, a.nmat, a.B, out.alpha, out.scat,
                                                          out.wdiff, out.wspec, out.thr, d_status);
        RP_TRY(cudaGetLastError());
        RP_TRY(cudaStreamSynchronize(st));
    }
done:
    cudaFree(blo); cudaFree(bhi); cudaFree(partial); cudaFree(bounds);
    cudaFree(k0); cudaFree(v0); cudaFree(k1); cudaFree(v1); cudaFree(hist);
    cudaFree(child); cudaFree(pint); cudaFree(pleaf); cudaFree(nn);
    for (int b = 0; b < 2; ++b) {
        cudaFree(cref[b]);
        cudaFree(clo[b]);
        cudaFree(chi[b]);
    }
    cudaFree(keep); cudaFree(kpos); cudaFree(merge); cudaFree(mpos);
    cudaFree(nlo); cudaFree(nhi); cudaFree(depth);
    return err;
}

}  // namespace rp
