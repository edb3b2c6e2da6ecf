// traverse.cuh -- BVH traversal for closest-hit and any-hit (shadow) queries.
//
// Stack-based while-while traversal in the style of Aila & Laine (HPG 2009): each
// node fetch is four 16-byte loads through the read-only path; both children's boxes
// are slab-tested together; leaf children (one triangle each) are intersected as soon
// as their box is hit; of two internal children the nearer is visited first and the
// farther is pushed.  The stack keeps its first SMEM_STACK entries in shared memory
// (one column per thread, conflict-free) and the rest in a small per-thread array.
//
// Closest hit: the nearest t in (tmin, tmax); equal t goes to the smaller original
// triangle index.  Any hit: some triangle with tmin < t < tmax.  The triangle
// `exclude` (leaf order) is skipped, which keeps a ray from re-hitting the surface
// it leaves.  Triangle test: Moller-Trumbore, two-sided, in FP32.
#pragma once

#include "internal.cuh"

namespace rp {

constexpr int SMEM_STACK = 24;
constexpr int LOCAL_STACK = 40;
constexpr int STACK_DEPTH = SMEM_STACK + LOCAL_STACK;
constexpr int ITER_CAP_MULT = 4;  // node visits per query are capped at 4 x nodes + 64

struct TravStats {
    uint32_t nodes;
    uint32_t tris;
};

__device__ __forceinline__ bool tri_intersect(const float4 *__restrict__ tris, int i, float3 o, float3 d,
                                              float &t, uint32_t &orig)
{
    const float4 a = __ldg(tris + 3 * i), b = __ldg(tris + 3 * i + 1), c = __ldg(tris + 3 * i + 2);
    const float3 e1 = xyz(b) - xyz(a), e2 = xyz(c) - xyz(a);
    const float3 p = cross(d, e2);
    const float det = dot(e1, p);
    if (det == 0.0f) return false;
    const float inv = 1.0f / det;
    const float3 s = o - xyz(a);
    const float u = dot(s, p) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    const float3 q = cross(s, e1);
    const float v = dot(d, q) * inv;
    if (v < 0.0f || u + v > 1.0f) return false;
    t = dot(e2, q) * inv;
    orig = __float_as_uint(b.w);
    return true;
}

template <bool ANY, bool COUNT>
__device__ __forceinline__ int traverse(const SceneView &sc, float3 o, float3 d, float tmin, float tmax,
                                        int exclude, int *__restrict__ sstack, float &t_out, TravStats &ts,
                                        int *status)
{
    const int stride = blockDim.x;
    int lstack[LOCAL_STACK];
    const float ex = fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x);
    const float ey = fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y);
    const float ez = fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z);
    const float3 idir = mk3(1.0f / ex, 1.0f / ey, 1.0f / ez);
    const float3 ood = mk3(o.x * idir.x, o.y * idir.y, o.z * idir.z);

    int best = -1;
    uint32_t best_orig = 0xffffffffu;
    float best_t = tmax;

    auto leaf = [&](int tri) -> bool {
        if (COUNT) ts.tris++;
        if ((unsigned)tri >= (unsigned)sc.num_tris) {  // corrupt structure: record, skip
            raise_error(status, RP_ERR_INVALID_ARG);
            return false;
        }
        float t;
        uint32_t orig;
        if (tri != exclude && tri_intersect(sc.tris, tri, o, d, t, orig) && t > tmin) {
            if (ANY) {
                if (t < tmax) {
                    best = tri;
                    best_t = t;
                    return true;
                }
            } else if (t < best_t || (t == best_t && best >= 0 && orig < best_orig)) {
                best = tri;
                best_t = t;
                best_orig = orig;
            }
        }
        return false;
    };

    if (sc.num_nodes == 0) {
        if (sc.num_tris > 0) leaf(0);
        t_out = best_t;
        return best;
    }

    const int iter_cap = ITER_CAP_MULT * sc.num_nodes + 64;
    int node = 0, sp = 0, iters = 0;
    while (true) {
        if (COUNT) ts.nodes++;
        if (++iters > iter_cap) {
            raise_error(status, RP_ERR_TIMEOUT);
            break;
        }
        if ((unsigned)node >= (unsigned)sc.num_nodes) {  // corrupt structure: record, stop
            raise_error(status, RP_ERR_INVALID_ARG);
            break;
        }
        const float4 *np = sc.nodes + 4 * node;
        const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
        const float a0 = n0.x * idir.x - ood.x, b0 = n0.y * idir.x - ood.x;
        const float a1 = n0.z * idir.y - ood.y, b1 = n0.w * idir.y - ood.y;
        const float a2 = n2.x * idir.z - ood.z, b2 = n2.y * idir.z - ood.z;
        const float c0min = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fmaxf(fminf(a2, b2), tmin));
        const float c0max = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fminf(fmaxf(a2, b2), best_t));
        const float a3 = n1.x * idir.x - ood.x, b3 = n1.y * idir.x - ood.x;
        const float a4 = n1.z * idir.y - ood.y, b4 = n1.w * idir.y - ood.y;
        const float a5 = n2.z * idir.z - ood.z, b5 = n2.w * idir.z - ood.z;
        const float c1min = fmaxf(fmaxf(fminf(a3, b3), fminf(a4, b4)), fmaxf(fminf(a5, b5), tmin));
        const float c1max = fminf(fminf(fmaxf(a3, b3), fmaxf(a4, b4)), fminf(fmaxf(a5, b5), best_t));
        bool h0 = c0min <= c0max, h1 = c1min <= c1max;
        const int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
        if (h0 && ch0 < 0) {
            if (leaf(~ch0)) break;
            h0 = false;
        }
        if (h1 && ch1 < 0) {
            if (leaf(~ch1)) break;
            h1 = false;
        }
        if (h0 && h1) {
            const bool swap = c1min < c0min;
            const int nearc = swap ? ch1 : ch0, farc = swap ? ch0 : ch1;
            if (sp < SMEM_STACK) {
                sstack[sp * stride] = farc;
            } else if (sp < STACK_DEPTH) {
                lstack[sp - SMEM_STACK] = farc;
            } else {
                raise_error(status, RP_ERR_STACK_OVERFLOW);
                break;
            }
            ++sp;
            node = nearc;
        } else if (h0) {
            node = ch0;
        } else if (h1) {
            node = ch1;
        } else {
            if (sp == 0) break;
            --sp;
            node = sp < SMEM_STACK ? sstack[sp * stride] : lstack[sp - SMEM_STACK];
        }
    }
    t_out = best_t;
    return best;
}

}  // namespace rp
