// refit.cu -- dynamic scenes: new vertex positions for an existing scene (the paper's
// scenes have moving objects, Section 6; its premise is interactive propagation in
// dynamic scenes) with the BVH refitted on the device instead of rebuilt.
//
// The tree keeps its topology.  One launch recomputes every box bottom-up: a thread
// per leaf writes its triangle (new vertices) and its box, then climbs: at each
// internal node the first of the two arriving threads stops and the second (it sees
// both children's boxes, ordered by a device-scope fence and an atomic counter per
// node) writes the node's padded child boxes and split code and goes on to the
// parent.  Child boxes are kept unpadded in a scratch array, so the padding does not
// grow with the depth.  The scene bounds, the box padding and the self-intersection
// guard follow from the new positions exactly as a build computes them.
#include <cmath>

#include "handles.cuh"

namespace rp {
namespace {

constexpr int RF_THREADS = 256;

// per-block min / max of the vertices: partial[blk][0..5] = (lo.xyz, hi.xyz); a
// non-finite coordinate raises RP_ERR_NAN_INPUT
__global__ void k_refit_bounds(const float *__restrict__ v, int nv, float *__restrict__ partial, int *status)
{
    __shared__ float s[6][RF_THREADS];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            const float x = v[3 * i + k];
            if (!isfinite(x)) raise_error(status, RP_ERR_NAN_INPUT);
            lo[k] = fminf(lo[k], x);
            hi[k] = fmaxf(hi[k], x);
        }
    }
    for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = lo[k];
        s[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int o = RF_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) {
                s[k][threadIdx.x] = fminf(s[k][threadIdx.x], s[k][threadIdx.x + o]);
                s[3 + k][threadIdx.x] = fmaxf(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) partial[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__device__ __forceinline__ float4 ld_box(const float4 *p) { return __ldcg(p); }

// one thread per leaf (Morton order): its triangle and box, then the climb
__global__ void k_refit(int nt, const float *__restrict__ verts, const int32_t *__restrict__ vidx,
                        float4 *__restrict__ tris, float4 *__restrict__ nodes, const int *__restrict__ pleaf,
                        const int *__restrict__ pint, float4 *__restrict__ bx_lo, float4 *__restrict__ bx_hi,
                        unsigned *__restrict__ arrivals, float pad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const float4 t0 = tris[3 * i], t1 = tris[3 * i + 1];
    const int orig = __float_as_int(t1.w);
    float3 p[3];
    for (int k = 0; k < 3; ++k) {
        const int vi = vidx[3 * orig + k];
        p[k] = mk3(verts[3 * vi], verts[3 * vi + 1], verts[3 * vi + 2]);
    }
    tris[3 * i] = make_float4(p[0].x, p[0].y, p[0].z, t0.w);
    tris[3 * i + 1] = make_float4(p[1].x, p[1].y, p[1].z, t1.w);
    tris[3 * i + 2] = make_float4(p[2].x, p[2].y, p[2].z, 0.f);
    if (nt < 2) return;
    // leaf boxes at [nt - 1 + i], internal nodes' at [node]
    bx_lo[nt - 1 + i] = make_float4(fminf(fminf(p[0].x, p[1].x), p[2].x), fminf(fminf(p[0].y, p[1].y), p[2].y),
                                    fminf(fminf(p[0].z, p[1].z), p[2].z), 0.f);
    bx_hi[nt - 1 + i] = make_float4(fmaxf(fmaxf(p[0].x, p[1].x), p[2].x), fmaxf(fmaxf(p[0].y, p[1].y), p[2].y),
                                    fmaxf(fmaxf(p[0].z, p[1].z), p[2].z), 0.f);
    int node = pleaf[i];
    for (int guard = 0; node >= 0 && guard < nt; ++guard) {
        __threadfence();  // this child's box is visible before the arrival is counted
        if (atomicAdd(&arrivals[node], 1u) == 0u) return;  // the sibling's thread finishes the node
        __threadfence();
        const float4 n3 = nodes[4 * node + 3];
        const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        const int s0 = c0 < 0 ? nt - 1 + ~c0 : c0, s1 = c1 < 0 ? nt - 1 + ~c1 : c1;
        const float4 l0 = ld_box(bx_lo + s0), h0 = ld_box(bx_hi + s0);
        const float4 l1 = ld_box(bx_lo + s1), h1 = ld_box(bx_hi + s1);
        nodes[4 * node + 0] = make_float4(l0.x - pad, h0.x + pad, l0.y - pad, h0.y + pad);
        nodes[4 * node + 1] = make_float4(l1.x - pad, h1.x + pad, l1.y - pad, h1.y + pad);
        nodes[4 * node + 2] = make_float4(l0.z - pad, h0.z + pad, l1.z - pad, h1.z + pad);
        // split code as the build makes it: the axis of the largest centre distance of
        // the children and whether the first child's centre is the higher one on it
        const float d[3] = {(l1.x + h1.x) - (l0.x + h0.x), (l1.y + h1.y) - (l0.y + h0.y),
                            (l1.z + h1.z) - (l0.z + h0.z)};
        const float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
        const int axis = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
        nodes[4 * node + 3] = make_float4(n3.x, n3.y, __int_as_float(axis | (d[axis] < 0.f ? 4 : 0)), n3.w);
        bx_lo[node] = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
        bx_hi[node] = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
        node = pint[node];
    }
}

}  // namespace
}  // namespace rp

using namespace rp;

extern "C" int rp_scene_refit(rp_scene *sc, const float *verts, int32_t num_verts, int32_t memory)
{
    if (!sc || !verts || num_verts != sc->num_verts || (memory != RP_MEM_HOST && memory != RP_MEM_DEVICE))
        return RP_ERR_INVALID_ARG;
    if (!sc->vidx || (sc->num_tris > 1 && (!sc->pleaf || !sc->pint))) return RP_ERR_INVALID_ARG;
    rp_ctx *c = sc->ctx;
    if (cudaSetDevice(c->device) != cudaSuccess) return RP_ERR_CUDA;
    cudaStream_t st = c->stream;
    const int nv = num_verts, nt = sc->num_tris;
    const int nblk = std::max(1, std::min(1024, (nv + RF_THREADS - 1) / RF_THREADS));
    float *dverts = nullptr, *partial = nullptr;
    float4 *blo = nullptr, *bhi = nullptr;
    unsigned *arrivals = nullptr;
    int rc = RP_OK;
    float hp[1024 * 6];
    cudaError_t e = cudaSuccess;
    const float *dv = verts;
    if (memory == RP_MEM_HOST) {
        if ((e = cudaMalloc(&dverts, sizeof(float) * 3 * nv)) == cudaSuccess)
            e = cudaMemcpyAsync(dverts, verts, sizeof(float) * 3 * nv, cudaMemcpyHostToDevice, st);
        dv = dverts;
    }
    if (e == cudaSuccess) e = cudaMalloc(&partial, sizeof(float) * 6 * nblk);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_refit_bounds<<<nblk, RF_THREADS, 0, st>>>(dv, nv, partial, c->d_status);
        e = cudaMemcpyAsync(hp, partial, sizeof(float) * 6 * nblk, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? RP_ERR_OOM : RP_ERR_CUDA;
        goto done;
    }
    if ((rc = rp_sync_status(c)) != RP_OK) goto done;  // non-finite vertices: the scene is left as it was
    {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int b = 0; b < nblk; ++b)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::fmin(lo[k], hp[6 * b + k]);
                hi[k] = std::fmax(hi[k], hp[6 * b + 3 + k]);
            }
        // bounds, padding and t_min as the build derives them (bvh.cu)
        float diag2 = 0.f, amax = 0.f;
        double dd2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            const float ext = hi[k] - lo[k];
            diag2 += ext * ext;
            amax = std::fmax(amax, std::fmax(std::fabs(lo[k]), std::fabs(hi[k])));
            dd2 += ((double)hi[k] - lo[k]) * ((double)hi[k] - lo[k]);
            sc->lo[k] = lo[k];
            sc->hi[k] = hi[k];
        }
        const float pad = 1e-6f * (amax + std::sqrt(diag2)) + 1e-30f;
        if (!(sc->ray_eps > 0.f)) {
            sc->tmin_d = 1e-6 * std::sqrt(dd2);
            sc->tmin = (float)sc->tmin_d;
        }
        if (nt > 1) {
            if ((e = cudaMalloc(&blo, sizeof(float4) * (2 * (size_t)nt - 1))) != cudaSuccess ||
                (e = cudaMalloc(&bhi, sizeof(float4) * (2 * (size_t)nt - 1))) != cudaSuccess ||
                (e = cudaMalloc(&arrivals, sizeof(unsigned) * (size_t)(nt - 1))) != cudaSuccess ||
                (e = cudaMemsetAsync(arrivals, 0, sizeof(unsigned) * (size_t)(nt - 1), st)) != cudaSuccess) {
                rc = e == cudaErrorMemoryAllocation ? RP_ERR_OOM : RP_ERR_CUDA;
                goto done;
            }
        }
        cudaEvent_t e0 = get_event(c), e1 = get_event(c);
        cudaEventRecord(e0, st);
        k_refit<<<(nt + RF_THREADS - 1) / RF_THREADS, RF_THREADS, 0, st>>>(nt, dv, sc->vidx, sc->tris, sc->nodes,
                                                                            sc->pleaf, sc->pint, blo, bhi, arrivals,
                                                                            pad);
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) cudaEventElapsedTime(&sc->refit_ms, e0, e1);
        c->free_events.push_back(e0);
        c->free_events.push_back(e1);
        if (e != cudaSuccess) rc = RP_ERR_CUDA;
    }
done:
    cudaFree(dverts);
    cudaFree(partial);
    cudaFree(blo);
    cudaFree(bhi);
    cudaFree(arrivals);
    return rc;
}
