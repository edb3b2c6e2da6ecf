// traverse.cuh -- BVH traversal for closest-hit and any-hit (shadow) queries.
//
// Stack-based while-while traversal in the style of Aila & Laine (HPG 2009): each
// node fetch is four 16-byte loads through the read-only path; both children's boxes
// are slab-tested together; leaf children (one triangle each) are intersected as soon
// as their box is hit; of two internal children a closest-hit query visits the nearer
// first, a resumable shadow-ray query (any_hit_steps) the one it enters later, and the
// other is pushed.  The stack keeps its first SMEM_STACK entries in shared memory
// (one column per thread, conflict-free) and the rest in a small per-thread array.
//
// Closest hit: the nearest t in (tmin, tmax); equal t goes to the smaller original
// triangle index.  In the FP64 decision (traverse_exact) "equal" means within TIE_REL
// (relative): coplanar overlapping surfaces meet a ray at one distance whose computed
// values differ only by rounding.  Any hit: some triangle with tmin < t < tmax.  The triangle
// `exclude` (leaf order) is skipped, which keeps a ray from re-hitting the surface
// it leaves.  Triangle test: Moller-Trumbore, two-sided.
//
// Precision: boxes and triangles are tested in FP32.  A query can ask to be told
// when its answer may depend on FP32 rounding -- a tested triangle lay within
// AMBIG_BARY (barycentric) of an edge at a distance that could decide the answer,
// or a hit lay within a relative AMBIG_T of t_min.  Such queries are re-run by
// traverse_exact(), whose triangle tests are FP64 on the FP64 ray; its box tests stay
// FP32 on the rounded ray, which the padding of the boxes keeps conservative.
#pragma once

#include "internal.cuh"

namespace rp {

constexpr int SMEM_STACK = 24;
constexpr int LOCAL_STACK = 40;
constexpr int STACK_DEPTH = SMEM_STACK + LOCAL_STACK;
constexpr float AMBIG_BARY = 2e-4f;
constexpr float AMBIG_T = 2e-4f;
constexpr double TIE_REL = 1e-9;  // FP64 closest-hit distances this close (relative) are equal

struct TravStats {
    uint32_t nodes;
    uint32_t tris;
    uint32_t walks = 0, steps = 0;  // shadow-ray packets: BVH walks and their node fetches (lane 0)
};

struct D3 {
    double x, y, z;
};

// Entry and exit distances of a ray through an axis-aligned box, from the distances
// (a_i, b_i) to the box's two planes on each axis: the largest of the per-axis minima
// and `lo`, and the smallest of the per-axis maxima and `hi`.  The three-input min and
// max of sm_100 and later take five operations for each instead of six.  The plane
// distances are finite (direction components are kept away from zero), so min and max
// return one of their inputs and the decisions match the two-input form exactly.
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float slab_in(float a0, float b0, float a1, float b1, float a2, float b2, float lo)
{
    return max3f(fminf(a0, b0), fminf(a1, b1), fmaxf(fminf(a2, b2), lo));
}

__device__ __forceinline__ float slab_out(float a0, float b0, float a1, float b1, float a2, float b2, float hi)
{
    return min3f(fmaxf(a0, b0), fmaxf(a1, b1), fminf(fmaxf(a2, b2), hi));
}

// FP32 Moller-Trumbore: t, the signed barycentric margin min(u, v, 1-u-v)
// (negative outside), and whether the ray passes inside the triangle.
__device__ __forceinline__ bool tri_intersect(const float4 *__restrict__ tris, int i, float3 o, float3 d,
                                              float &t, uint32_t &orig, float &margin)
{
    const float4 a = __ldg(tris + 3 * i), b = __ldg(tris + 3 * i + 1), c = __ldg(tris + 3 * i + 2);
    const float3 e1 = xyz(b) - xyz(a), e2 = xyz(c) - xyz(a);
    const float3 p = cross(d, e2);
    const float det = dot(e1, p);
    if (det == 0.0f) {
        margin = -1.0f;
        t = -1.0f;
        return false;
    }
    const float inv = 1.0f / det;
    const float3 s = o - xyz(a);
    const float u = dot(s, p) * inv;
    const float3 q = cross(s, e1);
    const float v = dot(d, q) * inv;
    t = dot(e2, q) * inv;
    orig = __float_as_uint(b.w);
    margin = fminf(fminf(u, v), 1.0f - u - v);
    return u >= 0.0f && u <= 1.0f && v >= 0.0f && u + v <= 1.0f;
}

// FP64 Moller-Trumbore on the exact input vertices (the FP64 reference test)
__device__ __forceinline__ bool tri_intersect_d(const float4 *__restrict__ tris, int i, D3 o, D3 d, double &t,
                                                uint32_t &orig)
{
    const float4 a = __ldg(tris + 3 * i), b = __ldg(tris + 3 * i + 1), c = __ldg(tris + 3 * i + 2);
    const double e1x = (double)b.x - a.x, e1y = (double)b.y - a.y, e1z = (double)b.z - a.z;
    const double e2x = (double)c.x - a.x, e2y = (double)c.y - a.y, e2z = (double)c.z - a.z;
    const double px = d.y * e2z - d.z * e2y, py = d.z * e2x - d.x * e2z, pz = d.x * e2y - d.y * e2x;
    const double det = e1x * px + e1y * py + e1z * pz;
    if (det == 0.0) return false;
    const double inv = 1.0 / det;
    const double sx = o.x - a.x, sy = o.y - a.y, sz = o.z - a.z;
    const double u = (sx * px + sy * py + sz * pz) * inv;
    if (u < 0.0 || u > 1.0) return false;
    const double qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
    const double v = (d.x * qx + d.y * qy + d.z * qz) * inv;
    if (v < 0.0 || u + v > 1.0) return false;
    t = (e2x * qx + e2y * qy + e2z * qz) * inv;
    orig = __float_as_uint(b.w);
    return true;
}

// Shared traversal loop.  `bound` is the current far limit of the query (the best
// hit so far, or tmax); leaf(tri) tests one triangle, may lower `bound`, and returns
// true to stop the query.
template <bool COUNT, typename Leaf>
__device__ __forceinline__ void traverse_core(const SceneView &sc, float3 o, float3 d, float tmin, float &bound,
                                              int *__restrict__ sstack, TravStats &ts, int *status, Leaf leaf)
{
    const int stride = blockDim.x;
    int lstack[LOCAL_STACK];
    const float ex = fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x);
    const float ey = fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y);
    const float ez = fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z);
    const float3 idir = mk3(1.0f / ex, 1.0f / ey, 1.0f / ez);
    const float3 ood = mk3(o.x * idir.x, o.y * idir.y, o.z * idir.z);

    if (sc.num_nodes == 0) {
        if (sc.num_tris > 0) {
            if (COUNT) ts.tris++;
            leaf(0);
        }
        return;
    }
    const int iter_cap = sc.iter_cap;
    int node = 0, sp = 0, iters = 0;
    while (true) {
        if (COUNT) ts.nodes++;
        if (++iters > iter_cap) {
            raise_error(status, RP_ERR_TIMEOUT);
            return;
        }
        if ((unsigned)node >= (unsigned)sc.num_nodes) {  // corrupt structure: record, stop
            raise_error(status, RP_ERR_INVALID_ARG);
            return;
        }
        const float4 *np = sc.nodes + 4 * node;
        const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
        const float a0 = n0.x * idir.x - ood.x, b0 = n0.y * idir.x - ood.x;
        const float a1 = n0.z * idir.y - ood.y, b1 = n0.w * idir.y - ood.y;
        const float a2 = n2.x * idir.z - ood.z, b2 = n2.y * idir.z - ood.z;
        const float c0min = slab_in(a0, b0, a1, b1, a2, b2, tmin);
        const float c0max = slab_out(a0, b0, a1, b1, a2, b2, bound);
        const float a3 = n1.x * idir.x - ood.x, b3 = n1.y * idir.x - ood.x;
        const float a4 = n1.z * idir.y - ood.y, b4 = n1.w * idir.y - ood.y;
        const float a5 = n2.z * idir.z - ood.z, b5 = n2.w * idir.z - ood.z;
        const float c1min = slab_in(a3, b3, a4, b4, a5, b5, tmin);
        const float c1max = slab_out(a3, b3, a4, b4, a5, b5, bound);
        bool h0 = c0min <= c0max, h1 = c1min <= c1max;
        const int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
        if (h0 && ch0 < 0) {
            const int tri = ~ch0;
            if (COUNT) ts.tris++;
            if ((unsigned)tri >= (unsigned)sc.num_tris) {
                raise_error(status, RP_ERR_INVALID_ARG);
                return;
            }
            if (leaf(tri)) return;
            h0 = false;
        }
        if (h1 && ch1 < 0) {
            const int tri = ~ch1;
            if (COUNT) ts.tris++;
            if ((unsigned)tri >= (unsigned)sc.num_tris) {
                raise_error(status, RP_ERR_INVALID_ARG);
                return;
            }
            if (leaf(tri)) return;
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
                return;
            }
            ++sp;
            node = nearc;
        } else if (h0) {
            node = ch0;
        } else if (h1) {
            node = ch1;
        } else {
            if (sp == 0) return;
            --sp;
            node = sp < SMEM_STACK ? sstack[sp * stride] : lstack[sp - SMEM_STACK];
        }
    }
}

// FP32 query.  With FLAG, *ambiguous tells whether the answer may depend on rounding
// (then the caller re-runs it with traverse_exact).
template <bool ANY, bool COUNT, bool FLAG>
__device__ __forceinline__ int traverse(const SceneView &sc, float3 o, float3 d, float tmin, float tmax,
                                        int exclude, int *__restrict__ sstack, float &t_out, TravStats &ts,
                                        int *status, bool *ambiguous = nullptr)
{
    int best = -1;
    uint32_t best_orig = 0xffffffffu;
    float bound = tmax;
    float amb_t = INFINITY;  // nearest distance of a rounding-sensitive triangle test
    float second = INFINITY; // closest hit: the runner-up distance (near-ties are sensitive)
    bool clear = false;      // any-hit: a blocker whose test is not rounding-sensitive
    const float tlo = tmin * (1.0f - AMBIG_T), tnear = tmin * (1.0f + AMBIG_T);
    traverse_core<COUNT>(sc, o, d, tmin, bound, sstack, ts, status, [&](int tri) -> bool {
        if (tri == exclude) return false;
        float t, margin;
        uint32_t orig;
        const bool inside = tri_intersect(sc.tris, tri, o, d, t, orig, margin);
        if (FLAG && t > tlo && t < tmax * (1.0f + AMBIG_T) &&
            (fabsf(margin) < AMBIG_BARY || (inside && t < tnear)))
            amb_t = fminf(amb_t, t);
        if (!inside || !(t > tmin)) return false;
        if (ANY) {
            if (t < tmax) {
                best = tri;
                if (!FLAG || (fabsf(margin) >= AMBIG_BARY && t >= tnear)) {
                    clear = true;
                    return true;
                }
            }
            return false;
        }
        if (t < bound || (t == bound && best >= 0 && orig < best_orig)) {
            if (FLAG && best >= 0) second = fminf(second, bound);
            best = tri;
            bound = t;
            best_orig = orig;
        } else if (FLAG) {
            second = fminf(second, t);
        }
        return false;
    });
    if (FLAG && ambiguous) {
        if (ANY) *ambiguous = !clear && amb_t < INFINITY;
        else if (best < 0) *ambiguous = amb_t < INFINITY;  // a miss is sensitive only near a tested edge
        else *ambiguous = fminf(amb_t, second) <= bound * (1.0f + AMBIG_T) + tmin;
    }
    t_out = bound;
    return best;
}

// FP64 re-run of a query whose FP32 answer was rounding-sensitive: the same
// traversal, FP64 triangle tests on the FP64 ray, decisions as in the FP64
// reference.
template <bool ANY>
__device__ __noinline__ int traverse_exact(const SceneView &sc, D3 o, D3 d, double tmin, double tmax, int exclude,
                                           int *__restrict__ sstack, double &t_out, int *status)
{
    int best = -1;
    uint32_t best_orig = 0xffffffffu;
    double best_t = tmax;
    // culling in FP32: bound just above best_t, t_min halved (boxes are padded)
    float bound = tmax < 3.0e38 ? __double2float_ru(tmax) : INFINITY;
    TravStats ts = {0u, 0u};
    const float3 of = mk3((float)o.x, (float)o.y, (float)o.z), df = mk3((float)d.x, (float)d.y, (float)d.z);
    const float tminf = __double2float_rd(tmin) * 0.5f;
    traverse_core<false>(sc, of, df, tminf, bound, sstack, ts, status, [&](int tri) -> bool {
        if (tri == exclude) return false;
        double t;
        uint32_t orig;
        if (!tri_intersect_d(sc.tris, tri, o, d, t, orig) || !(t > tmin)) return false;
        if (ANY) {
            if (t < tmax) {
                best = tri;
                best_t = t;
                return true;
            }
            return false;
        }
        const double tol = best >= 0 ? TIE_REL * fabs(best_t) : 0.0;
        if (best < 0 ? t < best_t : (t < best_t - tol || (t <= best_t + tol && orig < best_orig))) {
            best = tri;
            best_t = t;
            best_orig = orig;
            bound = __double2float_ru(t * (1.0 + TIE_REL));  // a tied candidate just beyond t stays in reach
        }
        return false;
    });
    t_out = best_t;
    return best;
}

}  // namespace rp

namespace rp {

// ---------------------------------------------------------------------------
// Resumable any-hit query: the traversal state lives in registers and the
// caller's stack columns between calls, so that a warp can advance each lane's
// query a few nodes at a time and give a finished lane a new ray immediately
// (persistent threads with per-lane refill).  Same decisions as
// traverse<true, COUNT, FLAG>.
// ---------------------------------------------------------------------------
struct AnyRay {
    float3 o, idir, ood;
    float tmin, tmax;
    int exclude;
};

struct AnyState {
    int node;      // next node to visit, -1 when the stack is empty
    int sp;        // stack depth
    float amb_t;   // nearest rounding-sensitive triangle distance
    bool blocked;  // a blocker was found
    bool clear;    // ... and its test was not rounding-sensitive
};

__device__ __forceinline__ AnyRay make_any_ray(float3 o, float3 d, float tmin, float tmax, int exclude)
{
    AnyRay r;
    const float ex = fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x);
    const float ey = fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y);
    const float ez = fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z);
    r.o = o;
    r.idir = mk3(1.0f / ex, 1.0f / ey, 1.0f / ez);
    r.ood = mk3(o.x * r.idir.x, o.y * r.idir.y, o.z * r.idir.z);
    r.tmin = tmin;
    r.tmax = tmax;
    r.exclude = exclude;
    return r;
}

// advance the query by at most `budget` node visits; returns true when it is done
template <bool COUNT, bool FLAG>
__device__ __forceinline__ bool any_hit_steps(const SceneView &sc, const AnyRay &r, float3 d, AnyState &q,
                                              int *__restrict__ sstack, int *lstack, int budget, TravStats &ts,
                                              int *status)
{
    const int stride = blockDim.x;
    const float tlo = r.tmin * (1.0f - AMBIG_T), tnear = r.tmin * (1.0f + AMBIG_T);
    auto leaf = [&](int tri) -> bool {  // true: query finished
        if (COUNT) ts.tris++;
        if ((unsigned)tri >= (unsigned)sc.num_tris) {
            raise_error(status, RP_ERR_INVALID_ARG);
            return true;
        }
        if (tri == r.exclude) return false;
        float t, margin;
        uint32_t orig;
        const bool inside = tri_intersect(sc.tris, tri, r.o, d, t, orig, margin);
        if (FLAG && t > tlo && t < r.tmax * (1.0f + AMBIG_T) &&
            (fabsf(margin) < AMBIG_BARY || (inside && t < tnear)))
            q.amb_t = fminf(q.amb_t, t);
        if (!inside || !(t > r.tmin) || !(t < r.tmax)) return false;
        q.blocked = true;
        if (!FLAG || (fabsf(margin) >= AMBIG_BARY && t >= tnear)) {
            q.clear = true;
            return true;
        }
        return false;
    };
    if (sc.num_nodes == 0) {
        if (sc.num_tris > 0) leaf(0);
        return true;
    }
    for (int it = 0; it < budget; ++it) {
        if (q.node < 0) return true;
        if (COUNT) ts.nodes++;
        if ((unsigned)q.node >= (unsigned)sc.num_nodes) {
            raise_error(status, RP_ERR_INVALID_ARG);
            return true;
        }
        const float4 *np = sc.nodes + 4 * q.node;
        const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
        const float a0 = n0.x * r.idir.x - r.ood.x, b0 = n0.y * r.idir.x - r.ood.x;
        const float a1 = n0.z * r.idir.y - r.ood.y, b1 = n0.w * r.idir.y - r.ood.y;
        const float a2 = n2.x * r.idir.z - r.ood.z, b2 = n2.y * r.idir.z - r.ood.z;
        const float c0min = slab_in(a0, b0, a1, b1, a2, b2, r.tmin);
        const float c0max = slab_out(a0, b0, a1, b1, a2, b2, r.tmax);
        const float a3 = n1.x * r.idir.x - r.ood.x, b3 = n1.y * r.idir.x - r.ood.x;
        const float a4 = n1.z * r.idir.y - r.ood.y, b4 = n1.w * r.idir.y - r.ood.y;
        const float a5 = n2.z * r.idir.z - r.ood.z, b5 = n2.w * r.idir.z - r.ood.z;
        const float c1min = slab_in(a3, b3, a4, b4, a5, b5, r.tmin);
        const float c1max = slab_out(a3, b3, a4, b4, a5, b5, r.tmax);
        bool h0 = c0min <= c0max, h1 = c1min <= c1max;
        const int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
        if (h0 && ch0 < 0) {
            if (leaf(~ch0)) return true;
            h0 = false;
        }
        if (h1 && ch1 < 0) {
            if (leaf(~ch1)) return true;
            h1 = false;
        }
        if (h0 && h1) {
            // the child the ray enters later goes first: a shadow ray leaves a surface,
            // and what blocks it lies more often towards the source than around its origin
            const bool swap = c1min > c0min;
            const int first = swap ? ch1 : ch0, second = swap ? ch0 : ch1;
            if (q.sp < SMEM_STACK) {
                sstack[q.sp * stride] = second;
            } else if (q.sp < STACK_DEPTH) {
                lstack[q.sp - SMEM_STACK] = second;
            } else {
                raise_error(status, RP_ERR_STACK_OVERFLOW);
                return true;
            }
            ++q.sp;
            q.node = first;
        } else if (h0) {
            q.node = ch0;
        } else if (h1) {
            q.node = ch1;
        } else if (q.sp == 0) {
            q.node = -1;
            return true;
        } else {
            --q.sp;
            q.node = q.sp < SMEM_STACK ? sstack[q.sp * stride] : lstack[q.sp - SMEM_STACK];
        }
    }
    return q.node < 0;
}

}  // namespace rp
