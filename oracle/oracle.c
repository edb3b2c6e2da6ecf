/*
 * oracle.c -- plain, slow FP64 CPU oracle of the ray-parameterized reverberation
 * hot path (Schissler & Manocha, "Interactive Sound Rendering on Mobile Devices
 * using Ray-Parameterized Reverberation Filters").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or table with the CUDA implementation; the
 * two meet only through the seeded scene generator and the published definitions
 * they both restate (Philox4x32-10, real spherical harmonics).
 *
 * What it computes, in the paper's order:
 *   - backward path tracing from the listener with diffuse rain (next-event
 *     estimation) at every reflection (Section 5, "Sound Propagation");
 *   - a low-rate per-band energy histogram I(t) together with its spherical-
 *     harmonic projection X_lm(t) (Section 4.2 first paragraph, symbol table);
 *   - direct sound of each source (Section 5, reduced to a point source);
 *   - the per-band reverberation parameters of Section 4.2: RT60 by backward
 *     energy integration and a least-squares decay fit, its exponential smoothing
 *     (Eq. for RT60 smoothing), total intensity and reverberator gain
 *     (Eq. reverb_gain with I_reverb^total = RT60 / (6 ln 10)), predelay,
 *     direct-to-reverberant ratio, weighted average directivity (Section 4.1
 *     directional-loudness equation) and the mean free path statistic;
 *   - the segment budget with refill of unused segments (Section 5).
 *
 * Everything is double precision.  Decisions that turn a float into an integer
 * and that both implementations must take identically (the diffuse/specular
 * choice) use an integer threshold computed from the float inputs.
 *
 * Readings where the paper is silent are listed in the design notes of the
 * repository; each is marked "[reading]" at the point of use below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXB 8
#define ORC_MAXK 16
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11). */
/* Each round: two 32x32->64 multiplies of counter words 0 and 2 by the round  */
/* multipliers, hi halves xored with the other counter words and the key, then */
/* the key is bumped by the Weyl constants.                                    */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in [0,1): top 24 bits, exact in float and double [reading] */
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

static void draw(uint64_t ray, uint32_t scene_id, uint32_t bounce, uint64_t seed, uint32_t out[4])
{
    uint32_t ctr[4] = { (uint32_t)ray, scene_id, bounce, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics, orthonormal, Condon-Shortley phase, ACN index      */
/* k = l*l + l + m (Section 2 "Spherical Harmonics"; the sign convention is the */
/* one under which Section 4.1's x_max = normalize(-X11, -X1-1, X10) recovers   */
/* the arrival direction).  Evaluated by the associated-Legendre recurrence.    */
/* ------------------------------------------------------------------------- */
static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* P_l^m(x) with the Condon-Shortley phase, m >= 0 */
static double assoc_legendre(int l, int m, double x)
{
    double pmm = 1.0;
    double somx2 = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x)));
    double fact = 1.0;
    for (int i = 1; i <= m; ++i) {
        pmm *= -fact * somx2;
        fact += 2.0;
    }
    if (l == m) return pmm;
    double pmmp1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pmmp1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * x * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pmmp1;
        pmmp1 = pll;
    }
    return pll;
}

void orc_sh_eval(int order, const double dir[3], double *Y)
{
    double len = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    double x = dir[0] / len, y = dir[1] / len, z = dir[2] / len;
    double phi = atan2(y, x);
    for (int l = 0; l <= order; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, z);
            double v;
            if (m > 0) v = sqrt(2.0) * K * P * cos(am * phi);
            else if (m < 0) v = sqrt(2.0) * K * P * sin(am * phi);
            else v = K * P;
            Y[l * l + l + m] = v;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Ray / triangle: Moller-Trumbore, two-sided.  Returns 1 and t on a hit.      */
/* ------------------------------------------------------------------------- */
static void sub3(const double a[3], const double b[3], double r[3]) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

int orc_intersect_tri(const double o[3], const double d[3], const double v0[3], const double v1[3],
                      const double v2[3], double *t_out)
{
    double e1[3], e2[3], p[3], q[3], s[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v0, s);
    double u = dot3(s, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    cross3(s, e1, q);
    double v = dot3(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    *t_out = dot3(e2, q) * inv;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Scene: mesh, materials and (optionally) a median-split BVH.                 */
/* ------------------------------------------------------------------------- */
typedef struct {
    double lo[3], hi[3];
    int left, right;   /* children, -1 for a leaf */
    int first, count;  /* leaf triangle range in `order` */
} orc_node;

typedef struct {
    int nv, nt, nmat, B;
    double *v;      /* [nv*3] */
    int *tri;       /* [nt*3] */
    int *mat;       /* [nt] */
    double *alpha;  /* [nmat*B] */
    double *scat;   /* [nmat*B] */
    double *sbar;   /* [nmat] mean scattering */
    uint32_t *thr;  /* [nmat] diffuse threshold on the 24-bit uniform */
    double tmin;
    int use_bvh;
    orc_node *nodes;
    int nnodes;
    int *order;
    double pad;
} orc_scene;

static const orc_scene *g_sort_scene;
static int g_sort_axis;

static double centroid(const orc_scene *sc, int t, int a)
{
    const int *ix = sc->tri + 3 * t;
    return (sc->v[3 * ix[0] + a] + sc->v[3 * ix[1] + a] + sc->v[3 * ix[2] + a]) / 3.0;
}

static int cmp_centroid(const void *pa, const void *pb)
{
    int a = *(const int *)pa, b = *(const int *)pb;
    double ca = centroid(g_sort_scene, a, g_sort_axis), cb = centroid(g_sort_scene, b, g_sort_axis);
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (a > b) - (a < b);
}

static int build_node(orc_scene *sc, int first, int count)
{
    int id = sc->nnodes++;
    orc_node *n = &sc->nodes[id];
    for (int a = 0; a < 3; ++a) { n->lo[a] = INFINITY; n->hi[a] = -INFINITY; }
    double clo[3] = { INFINITY, INFINITY, INFINITY }, chi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int i = first; i < first + count; ++i) {
        int t = sc->order[i];
        for (int c = 0; c < 3; ++c) {
            const double *p = sc->v + 3 * sc->tri[3 * t + c];
            for (int a = 0; a < 3; ++a) {
                if (p[a] < n->lo[a]) n->lo[a] = p[a];
                if (p[a] > n->hi[a]) n->hi[a] = p[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            double c = centroid(sc, t, a);
            if (c < clo[a]) clo[a] = c;
            if (c > chi[a]) chi[a] = c;
        }
    }
    for (int a = 0; a < 3; ++a) { n->lo[a] -= sc->pad; n->hi[a] += sc->pad; }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    n->left = n->right = -1;
    n->first = first;
    n->count = count;
    if (count <= 4 || chi[axis] - clo[axis] <= 0.0) return id;
    g_sort_scene = sc;
    g_sort_axis = axis;
    qsort(sc->order + first, (size_t)count, sizeof(int), cmp_centroid);
    int half = count / 2;
    int l = build_node(sc, first, half);
    int r = build_node(sc, first + half, count - half);
    sc->nodes[id].left = l;
    sc->nodes[id].right = r;
    sc->nodes[id].count = 0;
    return id;
}

void orc_scene_destroy(orc_scene *sc);

orc_scene *orc_scene_create(const float *verts, int nv, const int *tris, int nt, const int *mat,
                            const float *alpha, const float *scat, int nmat, int B, double ray_eps,
                            int use_bvh)
{
    if (nv <= 0 || nt <= 0 || nmat <= 0 || B <= 0 || B > ORC_MAXB) return NULL;
    orc_scene *sc = (orc_scene *)calloc(1, sizeof(orc_scene));
    sc->nv = nv; sc->nt = nt; sc->nmat = nmat; sc->B = B;
    sc->v = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    sc->tri = (int *)malloc(sizeof(int) * 3 * (size_t)nt);
    sc->mat = (int *)malloc(sizeof(int) * (size_t)nt);
    sc->alpha = (double *)malloc(sizeof(double) * (size_t)nmat * B);
    sc->scat = (double *)malloc(sizeof(double) * (size_t)nmat * B);
    sc->sbar = (double *)malloc(sizeof(double) * (size_t)nmat);
    sc->thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nmat);
    double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int i = 0; i < 3 * nv; ++i) {
        sc->v[i] = (double)verts[i];
        if (sc->v[i] < lo[i % 3]) lo[i % 3] = sc->v[i];
        if (sc->v[i] > hi[i % 3]) hi[i % 3] = sc->v[i];
    }
    for (int i = 0; i < 3 * nt; ++i) {
        if (tris[i] < 0 || tris[i] >= nv) { orc_scene_destroy(sc); return NULL; }
        sc->tri[i] = tris[i];
    }
    for (int i = 0; i < nt; ++i) {
        if (mat[i] < 0 || mat[i] >= nmat) { orc_scene_destroy(sc); return NULL; }
        sc->mat[i] = mat[i];
    }
    for (int m = 0; m < nmat; ++m) {
        double sum = 0.0;
        for (int b = 0; b < B; ++b) {
            sc->alpha[m * B + b] = (double)alpha[m * B + b];
            sc->scat[m * B + b] = (double)scat[m * B + b];
            sum += (double)scat[m * B + b];
        }
        sc->sbar[m] = sum / (double)B;
        /* u < sbar  <=>  u24 < ceil(sbar * 2^24) for the 24-bit integer u24 */
        sc->thr[m] = (uint32_t)ceil(sc->sbar[m] * 16777216.0);
    }
    double diag = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                       (hi[2] - lo[2]) * (hi[2] - lo[2]));
    /* self-intersection guard: t_min = 1e-6 * scene diagonal unless given [reading] */
    sc->tmin = ray_eps > 0.0 ? ray_eps : 1e-6 * diag;
    sc->pad = 1e-9 * diag + 1e-12;
    sc->use_bvh = use_bvh;
    if (use_bvh) {
        sc->order = (int *)malloc(sizeof(int) * (size_t)nt);
        for (int i = 0; i < nt; ++i) sc->order[i] = i;
        sc->nodes = (orc_node *)malloc(sizeof(orc_node) * (size_t)(2 * nt));
        sc->nnodes = 0;
        build_node(sc, 0, nt);
    }
    return sc;
}

void orc_scene_destroy(orc_scene *sc)
{
    if (!sc) return;
    free(sc->v); free(sc->tri); free(sc->mat); free(sc->alpha); free(sc->scat);
    free(sc->sbar); free(sc->thr); free(sc->nodes); free(sc->order);
    free(sc);
}

double orc_scene_tmin(const orc_scene *sc) { return sc->tmin; }
int orc_scene_num_nodes(const orc_scene *sc) { return sc->nnodes; }

static int tri_hit(const orc_scene *sc, int t, const double o[3], const double d[3], double *th)
{
    const int *ix = sc->tri + 3 * t;
    return orc_intersect_tri(o, d, sc->v + 3 * ix[0], sc->v + 3 * ix[1], sc->v + 3 * ix[2], th);
}

/* closest-hit candidate update: the nearer t wins; a t within ORC_TIE (relative) of the
 * best is equal and goes to the smaller triangle id [reading].  Coplanar overlapping
 * surfaces meet a ray at one mathematical distance, and the FP64 values computed from
 * their different vertices differ only by rounding, so "equal" means equal up to it. */
#define ORC_TIE 1e-9
static void consider(int t, double th, double tmin, int exclude, int *best, double *best_t)
{
    if (t == exclude || !(th > tmin)) return;
    if (*best < 0) {
        if (th < *best_t) {
            *best_t = th;
            *best = t;
        }
        return;
    }
    const double tol = ORC_TIE * fabs(*best_t);
    if (th < *best_t - tol || (th <= *best_t + tol && t < *best)) {
        *best_t = th;
        *best = t;
    }
}

static int slab(const orc_node *n, const double o[3], const double d[3], double tmin, double tmax,
                double *tnear)
{
    double t0 = tmin, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < n->lo[a] || o[a] > n->hi[a]) return 0;
            continue;
        }
        double ta = (n->lo[a] - o[a]) / d[a];
        double tb = (n->hi[a] - o[a]) / d[a];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    *tnear = t0;
    return 1;
}

/* closest hit with tmin < t < tmax, skipping triangle `exclude`; returns triangle or -1 */
int orc_closest_hit(const orc_scene *sc, const double o[3], const double d[3], double tmin, double tmax,
                    int exclude, double *t_out)
{
    int best = -1;
    double best_t = tmax;
    if (!sc->use_bvh) {
        for (int t = 0; t < sc->nt; ++t) {
            double th;
            if (tri_hit(sc, t, o, d, &th)) consider(t, th, tmin, exclude, &best, &best_t);
        }
    } else {
        int stack[128];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const orc_node *n = &sc->nodes[stack[--sp]];
            double tn;
            /* a box is kept when it may hold a hit at t <= best_t (ties included) */
            if (!slab(n, o, d, tmin - sc->pad, best_t + sc->pad, &tn)) continue;
            if (n->left < 0) {
                for (int i = n->first; i < n->first + n->count; ++i) {
                    int t = sc->order[i];
                    double th;
                    if (tri_hit(sc, t, o, d, &th)) consider(t, th, tmin, exclude, &best, &best_t);
                }
            } else {
                stack[sp++] = n->left;
                stack[sp++] = n->right;
            }
        }
    }
    if (best >= 0) *t_out = best_t;
    return best;
}

/* 1 if any triangle other than `exclude` is hit with tmin < t < tmax */
int orc_any_hit(const orc_scene *sc, const double o[3], const double d[3], double tmin, double tmax,
                int exclude)
{
    if (!sc->use_bvh) {
        for (int t = 0; t < sc->nt; ++t) {
            double th;
            if (t != exclude && tri_hit(sc, t, o, d, &th) && th > tmin && th < tmax) return 1;
        }
        return 0;
    }
    int stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const orc_node *n = &sc->nodes[stack[--sp]];
        double tn;
        if (!slab(n, o, d, tmin - sc->pad, tmax + sc->pad, &tn)) continue;
        if (n->left < 0) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int t = sc->order[i];
                double th;
                if (t != exclude && tri_hit(sc, t, o, d, &th) && th > tmin && th < tmax) return 1;
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Tracing (Section 5): backward path tracing from the listener with diffuse   */
/* rain, binned into the low-rate SH energy histogram (Section 4.2).           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t num_rays;      /* N primary rays (wave 0) */
    int32_t max_order;     /* M reflections per path */
    int32_t sh_order;      /* n, K = (n+1)^2 */
    int32_t num_bins;      /* T histogram bins */
    int32_t min_order;     /* reflections below this order are not binned */
    double ir_rate_hz;     /* histogram sample rate */
    double speed_of_sound; /* c */
    double source_radius;  /* r_s of the source spheres seen after specular bounces */
    uint64_t seed;         /* Philox key */
    uint32_t scene_id;     /* Philox counter word 1 */
    int32_t budget_refill; /* re-spend unused segments on extra primaries */
    int64_t first_ray;     /* id of the first primary */
} orc_trace_params;

/* layout of the stats array (doubles) */
enum {
    ST_ESCAPED = 0, ST_ABSORBED = 8, ST_REMAINING = 16, ST_LATE = 24,
    ST_MFP_SUM = 32, ST_MFP_CNT = 33, ST_MFP_SUM_NP = 34, ST_MFP_CNT_NP = 35,
    ST_SEGMENTS = 36, ST_SHADOW = 37, ST_PRIMARIES = 38, ST_CONTRIB = 39, ST_SPHERE = 40,
    ST_WAVES = 41, ST_COUNT = 48
};

#define FNV_OFFSET 0xcbf29ce484222325ull
#define FNV_PRIME 0x100000001b3ull
static uint64_t fnv_u32(uint64_t h, uint32_t v)
{
    for (int i = 0; i < 4; ++i) {
        h ^= (v >> (8 * i)) & 0xffu;
        h *= FNV_PRIME;
    }
    return h;
}

static void add_contrib(const orc_trace_params *p, int B, int K, int S_idx, const double *e,
                        double arrival_len, const double *Y, double *H, double *st)
{
    int T = p->num_bins;
    double t = arrival_len / p->speed_of_sound;
    double binf = floor(t * p->ir_rate_hz);
    st[ST_CONTRIB] += 1.0;
    if (binf >= (double)T) {
        for (int b = 0; b < B; ++b) st[ST_LATE + b] += e[b];
        return;
    }
    int bin = (int)binf;
    for (int b = 0; b < B; ++b)
        for (int k = 0; k < K; ++k)
            H[(((size_t)S_idx * B + b) * K + k) * T + bin] += e[b] * Y[k];
}

/* optional per-segment record of one ray (debugging divergence): triangle, t,
 * origin and direction of every segment */
typedef struct {
    int *tri;
    double *t, *o, *d;
    int n;
} orc_ray_log;

/* Early-reflection paths (Section 5: the first orders go to the diffuse path cache,
 * with spherical-harmonic directivity per path).  One record per visible diffuse-rain
 * contribution of a reflection of order 1 .. min_order - 1:
 *   [0] source, [1] order, [2] triangle of reflection 1, [3] triangle of reflection 2
 *   (-1 for order 1), [4] path length to the listener through the source, [5] primary
 *   ray id, [6 .. 14) energy per band (the contribution of the histogram's diffuse
 *   rain, not divided by the number of primaries; zero past B), [14 .. 30) the SH
 *   basis of the path's arrival direction (its first segment), zero past K */
#define ORC_ER_REC 30
typedef struct {
    double *rec;
    int64_t cap, n;
} orc_er_sink;

static void trace_ray(const orc_scene *sc, const orc_trace_params *p, const double lis[3],
                      const double *src, int S, uint64_t rid, double *H, double *st, uint64_t *hash_out,
                      orc_ray_log *log, orc_er_sink *er)
{
    const int B = sc->B, K = (p->sh_order + 1) * (p->sh_order + 1);
    /* with an early-reflection sink only the early orders are followed */
    const int M = er ? (p->max_order < p->min_order - 1 ? p->max_order : p->min_order - 1) : p->max_order;
    int seq[2] = { -1, -1 };
    uint32_t r[4];
    /* primary direction uniform on the sphere from bounce-0 draws [reading] */
    draw(rid, p->scene_id, 0u, p->seed, r);
    double z = 1.0 - 2.0 * u01(r[0]);
    double rad = sqrt(fmax(0.0, 1.0 - z * z));
    double phi = 2.0 * ORC_PI * u01(r[1]);
    double d[3] = { rad * cos(phi), rad * sin(phi), z };
    /* the arrival direction of every contribution of this path is its first
     * segment's direction (the symbol table's "direction toward source along
     * propagation path") */
    double Y[ORC_MAXK];
    orc_sh_eval(p->sh_order, d, Y);
    double o[3] = { lis[0], lis[1], lis[2] };
    double w[ORC_MAXB];
    for (int b = 0; b < B; ++b) w[b] = 1.0;
    double Lpath = 0.0;
    int prev = -1, spec_prev = 0;
    uint64_t hash = FNV_OFFSET;
    st[ST_PRIMARIES] += 1.0;
    for (int h = 1; h <= M; ++h) {
        double t = INFINITY;
        int tri = orc_closest_hit(sc, o, d, sc->tmin, INFINITY, prev, &t);
        st[ST_SEGMENTS] += 1.0;
        if (log) {
            log->tri[log->n] = tri;
            log->t[log->n] = t;
            for (int a = 0; a < 3; ++a) { log->o[3 * log->n + a] = o[a]; log->d[3 * log->n + a] = d[a]; }
            log->n++;
        }
        if (spec_prev && h - 1 >= p->min_order) {
            /* specularly reflected source image: the source as a sphere of radius
             * r_s on the segment after a specular choice [reading] */
            double rs = p->source_radius;
            for (int s = 0; s < S; ++s) {
                double oc[3];
                sub3(o, src + 3 * s, oc);
                double bq = dot3(oc, d);
                double cq = dot3(oc, oc) - rs * rs;
                double disc = bq * bq - cq;
                if (disc < 0.0) continue;
                double ts = -bq - sqrt(disc);
                if (!(ts > sc->tmin) || (tri >= 0 && !(ts < t))) continue;
                double e[ORC_MAXB];
                for (int b = 0; b < B; ++b) e[b] = w[b] / (ORC_PI * rs * rs);
                st[ST_SPHERE] += 1.0;
                add_contrib(p, B, K, s, e, Lpath + ts, Y, H, st);
            }
        }
        hash = fnv_u32(hash, tri < 0 ? 0xffffffffu : (uint32_t)tri);
        if (tri < 0) {
            for (int b = 0; b < B; ++b) st[ST_ESCAPED + b] += w[b];
            break;
        }
        Lpath += t;
        if (h <= 2) seq[h - 1] = tri;
        double hp[3] = { o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2] };
        st[ST_MFP_SUM] += t;
        st[ST_MFP_CNT] += 1.0;
        if (h > 1) { st[ST_MFP_SUM_NP] += t; st[ST_MFP_CNT_NP] += 1.0; }
        /* geometric normal turned toward the arriving ray: two-sided surfaces [reading] */
        const int *ix = sc->tri + 3 * tri;
        double e1[3], e2[3], n[3];
        sub3(sc->v + 3 * ix[1], sc->v + 3 * ix[0], e1);
        sub3(sc->v + 3 * ix[2], sc->v + 3 * ix[0], e2);
        cross3(e1, e2, n);
        double nl = sqrt(dot3(n, n));
        for (int a = 0; a < 3; ++a) n[a] /= nl;
        if (dot3(n, d) > 0.0) for (int a = 0; a < 3; ++a) n[a] = -n[a];
        const int m = sc->mat[tri];
        const double *al = sc->alpha + (size_t)m * B;
        const double *sc_b = sc->scat + (size_t)m * B;
        /* absorption first, then diffuse rain [reading: order of the two steps] */
        for (int b = 0; b < B; ++b) {
            st[ST_ABSORBED + b] += w[b] * al[b];
            w[b] *= (1.0 - al[b]);
        }
        if (h >= p->min_order) {
            /* diffuse rain: one shadow ray per source; a visible source adds the
             * Lambertian reflection of its direct irradiance,
             * w_b * s_b * cos(theta) / (pi * d^2) per unit source power and ray */
            for (int s = 0; s < S; ++s) {
                double v[3];
                sub3(src + 3 * s, hp, v);
                double dist = sqrt(dot3(v, v));
                double cs = dot3(n, v) / dist;
                if (!(cs > 0.0)) continue;
                double dir[3] = { v[0] / dist, v[1] / dist, v[2] / dist };
                st[ST_SHADOW] += 1.0;
                if (orc_any_hit(sc, hp, dir, sc->tmin, dist, tri)) continue;
                double e[ORC_MAXB];
                for (int b = 0; b < B; ++b) e[b] = w[b] * sc_b[b] * cs / (ORC_PI * dist * dist);
                add_contrib(p, B, K, s, e, Lpath + dist, Y, H, st);
            }
        } else if (er && h <= 2) {
            /* an early reflection: the same diffuse rain, kept as a path record keyed
             * by the source and the reflections' triangles */
            for (int s = 0; s < S; ++s) {
                double v[3];
                sub3(src + 3 * s, hp, v);
                double dist = sqrt(dot3(v, v));
                double cs = dot3(n, v) / dist;
                if (!(cs > 0.0)) continue;
                double dir[3] = { v[0] / dist, v[1] / dist, v[2] / dist };
                if (orc_any_hit(sc, hp, dir, sc->tmin, dist, tri)) continue;
                if (er->n < er->cap) {
                    double *q = er->rec + (size_t)er->n * ORC_ER_REC;
                    q[0] = s;
                    q[1] = h;
                    q[2] = seq[0];
                    q[3] = h >= 2 ? seq[1] : -1.0;
                    q[4] = Lpath + dist;
                    q[5] = (double)rid;
                    for (int b = 0; b < ORC_MAXB; ++b) q[6 + b] = b < B ? w[b] * sc_b[b] * cs / (ORC_PI * dist * dist) : 0.0;
                    for (int k = 0; k < ORC_MAXK; ++k) q[14 + k] = k < K ? Y[k] : 0.0;
                }
                er->n++;
            }
        }
        if (h == M) {
            for (int b = 0; b < B; ++b) st[ST_REMAINING + b] += w[b];
            break;
        }
        /* continuation: diffuse with probability sbar (cosine-weighted hemisphere),
         * otherwise mirror reflection; weights keep the estimator unbiased per band */
        draw(rid, p->scene_id, (uint32_t)h, p->seed, r);
        if ((r[2] >> 8) < sc->thr[m]) {
            double u0 = u01(r[0]), u1 = u01(r[1]);
            double rr = sqrt(u1), ph = 2.0 * ORC_PI * u0;
            double lx = rr * cos(ph), ly = rr * sin(ph), lz = sqrt(fmax(0.0, 1.0 - u1));
            /* orthonormal frame around n: Duff et al. 2017 */
            double sg = n[2] >= 0.0 ? 1.0 : -1.0;
            double a = -1.0 / (sg + n[2]);
            double bb = n[0] * n[1] * a;
            double b1[3] = { 1.0 + sg * n[0] * n[0] * a, sg * bb, -sg * n[0] };
            double b2[3] = { bb, sg + n[1] * n[1] * a, -n[1] };
            for (int k = 0; k < 3; ++k) d[k] = lx * b1[k] + ly * b2[k] + lz * n[k];
            for (int b = 0; b < B; ++b) w[b] *= sc_b[b] / sc->sbar[m];
            spec_prev = 0;
        } else {
            double dn = dot3(d, n);
            for (int k = 0; k < 3; ++k) d[k] -= 2.0 * dn * n[k];
            double dl = sqrt(dot3(d, d));
            for (int k = 0; k < 3; ++k) d[k] /= dl;
            for (int b = 0; b < B; ++b) w[b] *= (1.0 - sc_b[b]) / (1.0 - sc->sbar[m]);
            spec_prev = 1;
        }
        o[0] = hp[0]; o[1] = hp[1]; o[2] = hp[2];
        prev = tri;
    }
    if (hash_out) *hash_out = hash;
}

/* Raw (un-normalised) histogram sums and stats for primary rays [ray_begin, ray_end).
 * H_raw [S][B][K][T] and stats[ST_COUNT] are accumulated into.  ray_hash, if not NULL,
 * receives one 64-bit FNV-1a hash of each ray's triangle sequence. */
void orc_trace_rays(const orc_scene *sc, const orc_trace_params *p, const double lis[3],
                    const double *src, int S, int64_t ray_begin, int64_t ray_end, double *H_raw,
                    double *st, uint64_t *ray_hash)
{
    for (int64_t r = ray_begin; r < ray_end; ++r)
        trace_ray(sc, p, lis, src, S, (uint64_t)r, H_raw, st, ray_hash ? &ray_hash[r - ray_begin] : NULL, NULL, NULL);
}

/* Early-reflection path records (ORC_ER_REC doubles each) of primaries
 * [ray_begin, ray_end): each path followed to order min_order - 1 (at most 2) with the
 * random numbers of the full trace.  Writes at most cap records; returns how many
 * there are. */
int64_t orc_er_rays(const orc_scene *sc, const orc_trace_params *p, const double lis[3], const double *src, int S,
                    int64_t ray_begin, int64_t ray_end, double *rec, int64_t cap)
{
    const int B = sc->B, K = (p->sh_order + 1) * (p->sh_order + 1);
    double st[ST_COUNT];
    double Hd[ORC_MAXB * ORC_MAXK];  /* never written: no order reaches min_order */
    orc_er_sink er = { rec, cap, 0 };
    (void)B;
    (void)K;
    for (int64_t r = ray_begin; r < ray_end; ++r) trace_ray(sc, p, lis, src, S, (uint64_t)r, Hd, st, NULL, NULL, &er);
    return er.n;
}

/* Debug: the segments of primary ray `rid` (at most max_order entries); returns
 * the number of segments.  H_raw and st receive the ray's contributions. */
int orc_trace_ray_log(const orc_scene *sc, const orc_trace_params *p, const double lis[3], const double *src,
                      int S, uint64_t rid, double *H_raw, double *st, int *tri, double *t, double *o, double *d)
{
    orc_ray_log log = { tri, t, o, d, 0 };
    trace_ray(sc, p, lis, src, S, rid, H_raw, st, NULL, &log, NULL);
    return log.n;
}

/* Direct sound of a point source (reduction of Section 5's direct-sound step):
 * visible if the listener-source segment is unoccluded; energy 1/(4 pi d^2),
 * arrival d/c, SH of the direction toward the source.
 * out per source: [visible, dist, time, energy, bin, sh[16]] (21 doubles). */
void orc_direct(const orc_scene *sc, const orc_trace_params *p, const double lis[3], const double *src,
                int S, double *out)
{
    for (int s = 0; s < S; ++s) {
        double v[3];
        sub3(src + 3 * s, lis, v);
        double dist = sqrt(dot3(v, v));
        double dir[3] = { v[0] / dist, v[1] / dist, v[2] / dist };
        int blocked = orc_any_hit(sc, lis, dir, sc->tmin, dist, -1);
        double *o = out + (size_t)s * 21;
        memset(o, 0, sizeof(double) * 21);
        o[0] = blocked ? 0.0 : 1.0;
        o[1] = dist;
        o[2] = dist / p->speed_of_sound;
        o[3] = blocked ? 0.0 : 1.0 / (4.0 * ORC_PI * dist * dist);
        o[4] = floor(o[2] * p->ir_rate_hz);
        double Y[ORC_MAXK];
        orc_sh_eval(p->sh_order, dir, Y);
        int K = (p->sh_order + 1) * (p->sh_order + 1);
        for (int k = 0; k < K; ++k) o[5 + k] = o[3] * Y[k];
    }
}

/* Number of primaries of the next wave under the segment budget of Section 5:
 * the budget is N*M segments; unused segments buy floor(unused / M) new rays. */
int64_t orc_next_wave(int64_t N, int M, double segments_used)
{
    double unused = (double)N * (double)M - segments_used;
    if (unused < (double)M) return 0;
    return (int64_t)floor(unused / (double)M);
}

/* The whole trace step: waves of primaries (one wave unless budget_refill),
 * normalisation by the number of primaries K, and direct sound binned into H
 * when min_order == 0.  H [S][B][K][T] is overwritten.  ray_hash[i] receives the
 * hash of ray first_ray + i for i < hash_cap. Returns the number of waves. */
int orc_trace(const orc_scene *sc, const orc_trace_params *p, const double lis[3], const double *src,
              int S, double *H, double *st, uint64_t *ray_hash, int64_t hash_cap)
{
    const int B = sc->B, K = (p->sh_order + 1) * (p->sh_order + 1), T = p->num_bins;
    size_t nH = (size_t)S * B * K * T;
    memset(H, 0, sizeof(double) * nH);
    memset(st, 0, sizeof(double) * ST_COUNT);
    int64_t begin = p->first_ray, count = p->num_rays;
    int waves = 0;
    while (count > 0 && waves < 4096) {
        for (int64_t r = begin; r < begin + count; ++r) {
            const int64_t hi = r - p->first_ray;
            uint64_t *hp = (ray_hash && hi >= 0 && hi < hash_cap) ? &ray_hash[hi] : NULL;
            trace_ray(sc, p, lis, src, S, (uint64_t)r, H, st, hp, NULL, NULL);
        }
        begin += count;
        waves++;
        count = p->budget_refill ? orc_next_wave(p->num_rays, p->max_order, st[ST_SEGMENTS]) : 0;
    }
    st[ST_WAVES] = waves;
    double kp = st[ST_PRIMARIES];
    if (kp > 0.0)
        for (size_t i = 0; i < nH; ++i) H[i] /= kp;
    for (int b = 0; b < B; ++b) st[ST_LATE + b] /= (kp > 0.0 ? kp : 1.0);
    if (p->min_order == 0) {
        double *dd = (double *)malloc(sizeof(double) * 21 * (size_t)S);
        orc_direct(sc, p, lis, src, S, dd);
        for (int s = 0; s < S; ++s) {
            double *o = dd + (size_t)s * 21;
            if (o[0] == 0.0) continue;
            if (o[4] >= (double)T) continue;
            int bin = (int)o[4];
            for (int b = 0; b < B; ++b)
                for (int k = 0; k < K; ++k)
                    H[(((size_t)s * B + b) * K + k) * T + bin] += o[5 + k];
        }
        free(dd);
    }
    return waves;
}

/* ------------------------------------------------------------------------- */
/* Reverberation parameter estimation (Section 4.2), per (source, band).       */
/* out per (s,b), 32 doubles:                                                  */
/*  0 rt60_raw  1 rt60_smoothed  2 fit_hi_db  3 fit_lo_db  4 fit_r2            */
/*  5 slope_db_per_s  6 intercept_db  7 i_total  8 g_reverb  9 e_direct        */
/* 10 drr_db  11 predelay_s  12 range_kind  13 n_fit  14 fit_j0  15 fit_j1     */
/* 16..31 xbar[16]                                                             */
/* range_kind: 0 none, 1 T30 (-5..-35 dB), 2 T20 (-5..-25), 3 T10 (0..-10)     */
/* ------------------------------------------------------------------------- */
#define EP_COUNT 32

void orc_estimate(const double *H, const double *e_direct, int S, int B, int K, int T, double ir_rate_hz,
                  double dt_update, double tau, double *out, double *state)
{
    static const double ranges[3][2] = { { -5.0, -35.0 }, { -5.0, -25.0 }, { 0.0, -10.0 } };
    const double sq4pi = sqrt(4.0 * ORC_PI);
    double *I = (double *)malloc(sizeof(double) * (size_t)T);
    double *E = (double *)malloc(sizeof(double) * (size_t)T);
    double *Ld = (double *)malloc(sizeof(double) * (size_t)T);
    double *isum = (double *)calloc((size_t)T, sizeof(double));
    for (int s = 0; s < S; ++s) {
        /* predelay: first bin that is non-zero in any band [reading of Section 4.2] */
        memset(isum, 0, sizeof(double) * (size_t)T);
        for (int b = 0; b < B; ++b)
            for (int j = 0; j < T; ++j) isum[j] += sq4pi * H[(((size_t)s * B + b) * K + 0) * T + j];
        int first = -1;
        for (int j = 0; j < T; ++j)
            if (isum[j] > 0.0) { first = j; break; }
        for (int b = 0; b < B; ++b) {
            double *o = out + ((size_t)s * B + b) * EP_COUNT;
            for (int i = 0; i < EP_COUNT; ++i) o[i] = 0.0;
            const double *h0 = H + (((size_t)s * B + b) * K + 0) * T;
            /* intensity histogram: I = sqrt(4 pi) * X_00 since Y_00 = 1/sqrt(4 pi) */
            for (int j = 0; j < T; ++j) I[j] = sq4pi * h0[j];
            /* backward (Schroeder) integration */
            double acc = 0.0;
            for (int j = T - 1; j >= 0; --j) { acc += I[j]; E[j] = acc; }
            double itot = 0.0;
            for (int j = 0; j < T; ++j) itot += I[j];
            o[7] = itot;
            double rt = NAN, slope = NAN, icpt = NAN, r2 = NAN;
            int kind = 0, nfit = 0, j0 = -1, j1 = -1;
            if (E[0] > 0.0) {
                for (int j = 0; j < T; ++j) Ld[j] = E[j] > 0.0 ? 10.0 * log10(E[j] / E[0]) : -INFINITY;
                for (int rk = 0; rk < 3 && kind == 0; ++rk) {
                    double hi = ranges[rk][0], lo = ranges[rk][1];
                    int n = 0, a = -1, z = -1, reached = 0;
                    for (int j = 0; j < T; ++j) {
                        if (Ld[j] <= hi && Ld[j] >= lo) { if (a < 0) a = j; z = j; n++; }
                        if (Ld[j] < lo) reached = 1;
                    }
                    if (n < 3 || !reached) continue;
                    /* least squares of level on bin start time */
                    double sx = 0, sy = 0;
                    for (int j = a; j <= z; ++j) { sx += j / ir_rate_hz; sy += Ld[j]; }
                    double mx = sx / n, my = sy / n, sxx = 0, sxy = 0, syy = 0;
                    for (int j = a; j <= z; ++j) {
                        double dx = j / ir_rate_hz - mx, dy = Ld[j] - my;
                        sxx += dx * dx; sxy += dx * dy; syy += dy * dy;
                    }
                    double sl = sxy / sxx;
                    if (!(sl < 0.0)) continue;
                    slope = sl;
                    icpt = my - sl * mx;
                    r2 = syy > 0.0 ? (sxy * sxy) / (sxx * syy) : 1.0;
                    rt = -60.0 / sl;
                    kind = rk + 1; nfit = n; j0 = a; j1 = z;
                    o[2] = hi; o[3] = lo;
                }
            }
            o[0] = rt; o[4] = r2; o[5] = slope; o[6] = icpt;
            o[12] = kind; o[13] = nfit; o[14] = j0; o[15] = j1;
            /* reverberator gain: I_reverb^total = RT60 / (6 ln 10), g = sqrt(I_total / I_reverb) */
            o[8] = (kind > 0 && itot >= 0.0) ? sqrt(itot / (rt / (6.0 * log(10.0)))) : NAN;
            double ed = e_direct ? e_direct[s] : 0.0;
            o[9] = ed;
            if (ed > 0.0 && itot > 0.0) o[10] = 10.0 * log10(ed / itot);
            else if (ed > 0.0) o[10] = INFINITY;
            else if (itot > 0.0) o[10] = -INFINITY;
            else o[10] = NAN;
            o[11] = first >= 0 ? first / ir_rate_hz : NAN;
            /* weighted average directivity: sum_t X_lm(t) / sum_t I(t) (X * I = H) */
            for (int k = 0; k < K && k < 16; ++k) {
                const double *hk = H + (((size_t)s * B + b) * K + k) * T;
                double sk = 0.0;
                for (int j = 0; j < T; ++j) sk += hk[j];
                o[16 + k] = itot > 0.0 ? sk / itot : NAN;
            }
            /* exponential smoothing: alpha = 1 - exp(-dt / tau) [reading] */
            double sm = rt;
            if (state) {
                double prev = state[(size_t)s * B + b];
                double alpha = tau > 0.0 ? 1.0 - exp(-dt_update / tau) : 1.0;
                if (isnan(prev)) sm = rt;
                else if (isnan(rt)) sm = prev;
                else sm = alpha * rt + (1.0 - alpha) * prev;
                state[(size_t)s * B + b] = sm;
            }
            o[1] = sm;
        }
    }
    free(I); free(E); free(Ld); free(isum);
}

/* mean free path (Section 4.2 "Reflection Density"): average length of the
 * segments that ended on a surface, primary segments included [reading] */
double orc_mean_free_path(const double *st) { return st[ST_MFP_CNT] > 0 ? st[ST_MFP_SUM] / st[ST_MFP_CNT] : NAN; }
