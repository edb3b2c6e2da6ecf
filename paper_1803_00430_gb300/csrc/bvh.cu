// bvh.cu -- device construction of the scene's bounding-volume hierarchy.
//
// The paper's ray tracer leaves its acceleration structure unspecified (Section 6
// "Performance" only states that cost grows logarithmically with scene size).  This
// file builds a linear BVH entirely on the GPU:
//   1. per-triangle bounds and centroids, checked for non-finite values;
//   2. 30-bit Morton codes of the centroids;
//   3. a stable LSD radix sort (8-bit digits) of (code, triangle) pairs;
//   4. the binary radix tree of Karras (HPG 2012), one thread per internal node,
//      with ties between equal codes broken by the leaf index;
//   5. bottom-up child bounds (one thread per leaf, the second arrival at a node
//      continues upward);
//   6. packing into 64-byte nodes holding both children's boxes, and 48-byte
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

// --- 4. Karras radix tree ------------------------------------------------------------
__device__ __forceinline__ int delta(const uint32_t *__restrict__ codes, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    const uint32_t a = codes[i], b = codes[j];
    if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clz(a ^ b);
}

__global__ void k_karras(const uint32_t *__restrict__ codes, int n, int2 *__restrict__ child,
                         int *__restrict__ parent_int, int *__restrict__ parent_leaf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(codes, n, i, i + 1) - delta(codes, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(codes, n, i, i - d);
    int lmax = 2;
    while (delta(codes, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(codes, n, i, j);
    int s = 0;
    int div = 2;
    int t = (l + div - 1) / div;
    while (true) {
        if (delta(codes, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
        div <<= 1;
        t = (l + div - 1) / div;
    }
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    int left, right;
    if (lo == gamma) {
        left = ~gamma;
        parent_leaf[gamma] = i;
    } else {
        left = gamma;
        parent_int[gamma] = i;
    }
    if (hi == gamma + 1) {
        right = ~(gamma + 1);
        parent_leaf[gamma + 1] = i;
    } else {
        right = gamma + 1;
        parent_int[gamma + 1] = i;
    }
    child[i] = make_int2(left, right);
}

// --- 5. bottom-up bounds ---------------------------------------------------------------
__device__ __forceinline__ void child_box(int c, const uint32_t *__restrict__ order,
                                          const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                                          const float4 *nlo, const float4 *nhi, float4 &lo, float4 &hi)
{
    if (c < 0) {
        const uint32_t t = order[~c];
        lo = blo[t];
        hi = bhi[t];
    } else {
        lo = __ldcg(nlo + c);
        hi = __ldcg(nhi + c);
    }
}

__global__ void k_bounds(int n, const uint32_t *__restrict__ order, const float4 *__restrict__ blo,
                         const float4 *__restrict__ bhi, const int2 *__restrict__ child,
                         const int *__restrict__ parent_int, const int *__restrict__ parent_leaf,
                         int *__restrict__ flags, float4 *nlo, float4 *nhi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = parent_leaf[i];
    int guard = 0;
    while (p >= 0 && p < n - 1 && guard++ < 4096) {
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;  // the sibling subtree finishes this node
        const int2 c = child[p];
        float4 l0, h0, l1, h1;
        child_box(c.x, order, blo, bhi, nlo, nhi, l0, h0);
        child_box(c.y, order, blo, bhi, nlo, nhi, l1, h1);
        __stcg(nlo + p, make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f));
        __stcg(nhi + p, make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f));
        if (p == 0) return;
        p = parent_int[p];
    }
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
    nodes[4 * i + 3] = make_float4(__int_as_float(c.x), __int_as_float(c.y), 0.f, 0.f);
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
    int *pint = nullptr, *pleaf = nullptr, *flags = nullptr, *depth = nullptr;
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
    RP_TRY(dalloc(&flags, nt));
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
    RP_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * nt, st));
    RP_TRY(cudaMemsetAsync(depth, 0, sizeof(int), st));
    if (nt > 1) {
        k_karras<<<(nt - 1 + 255) / 256, 256, 0, st>>>(k0, nt, child, pint, pleaf);
        k_bounds<<<nblk_tri, 256, 0, st>>>(nt, v0, blo, bhi, child, pint, pleaf, flags, nlo, nhi);
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
        k_materials<<<(a.nmat + 127) / 128, 128, 0, st>>>(a.alpha, a.scat, a.nmat, a.B, out.alpha, out.scat,
                                                          out.wdiff, out.wspec, out.thr, d_status);
        RP_TRY(cudaGetLastError());
        RP_TRY(cudaStreamSynchronize(st));
    }
done:
    cudaFree(blo); cudaFree(bhi); cudaFree(partial); cudaFree(bounds);
    cudaFree(k0); cudaFree(v0); cudaFree(k1); cudaFree(v1); cudaFree(hist);
    cudaFree(child); cudaFree(pint); cudaFree(pleaf); cudaFree(flags);
    cudaFree(nlo); cudaFree(nhi); cudaFree(depth);
    return err;
}

}  // namespace rp
