/*
 * rpr.h -- C ABI of the GB300 ray-parameterized reverberation library.
 *
 * The library computes, on one GPU, the sound-propagation and parameter-estimation
 * hot path of "Interactive Sound Rendering on Mobile Devices using
 * Ray-Parameterized Reverberation Filters" (Schissler & Manocha):
 *
 *   rp_scene_create  builds a bounding-volume hierarchy of the scene mesh on the
 *                    device (the paper's ray tracer, Section 6 "Performance", does
 *                    not describe its acceleration structure).
 *   rp_trace         backward path tracing from the listener with diffuse rain
 *                    (next-event estimation) at every reflection (Section 5, "Sound
 *                    Propagation"), binned into a low-rate energy impulse response
 *                    per source and band together with its spherical-harmonic
 *                    projection X_lm(t) (Section 4.2 first paragraph; Table of
 *                    symbols), plus direct sound (Section 5) and the mean free path
 *                    statistic (Section 4.2 "Reflection Density").
 *   rp_estimate      per-band reverberation parameters from those IRs (Section 4.2):
 *                    RT60 by backward energy integration and a least-squares decay
 *                    fit, its exponential smoothing (RT60 smoothing equation), total
 *                    intensity and reverberator gain (Eq. reverb_gain with
 *                    I_reverb^total = RT60 / (6 ln 10)), predelay, direct-to-
 *                    reverberant ratio and the weighted average directivity of
 *                    Section 4.1 ("Directional Loudness").
 *   rp_update        trace + estimate with host buffers (copies included).
 *
 * Conventions (all entry points):
 *   - Every call returns an int status: RP_OK (0) or a negative RP_ERR_* code.
 *     Nothing throws across the ABI.  rp_status_string() names a code.
 *   - Work is enqueued asynchronously on the context's CUDA stream.  Errors that
 *     kernels detect (capacity, traversal stack, iteration cap) are recorded in a
 *     device status word and returned by rp_sync_status(), which synchronises the
 *     stream.  Device pointers passed in must stay valid until then.
 *   - The caller owns every output buffer; the library owns rp_ctx and rp_scene
 *     objects and its internal workspace, released by the matching destroy call.
 *   - Arrays are dense, row-major, in the index order written next to them.
 *   - A context is not thread-safe: one host thread at a time per rp_ctx.
 *   - Limits: bands B <= RP_MAX_BANDS, SH order n <= RP_MAX_SH_ORDER
 *     (K = (n+1)^2 <= RP_MAX_SH), sources S <= RP_MAX_SOURCES.
 */
#ifndef RPR_H
#define RPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RP_MAX_BANDS 8
#define RP_MAX_SH_ORDER 3
#define RP_MAX_SH 16
#define RP_MAX_SOURCES 4096

enum {
    RP_OK = 0,
    RP_ERR_INVALID_ARG = -1,    /* a pointer, size or parameter is out of range */
    RP_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    RP_ERR_OOM = -3,            /* device memory allocation failed */
    RP_ERR_CAPACITY = -4,       /* an internal buffer overflowed; results incomplete */
    RP_ERR_STACK_OVERFLOW = -5, /* BVH traversal stack overflowed; results incomplete */
    RP_ERR_TIMEOUT = -6,        /* a traversal exceeded its iteration cap */
    RP_ERR_NAN_INPUT = -7,      /* a vertex, material or position is not finite */
    RP_ERR_EMPTY_SCENE = -8,    /* zero triangles */
    RP_ERR_NO_DEVICE = -9,      /* no CUDA device or wrong architecture */
    RP_ERR_TOO_LARGE = -10,     /* the problem does not fit the fixed scratch of
                                   rp_trace_noalloc (RP_NOALLOC_SCRATCH_BYTES) */
    RP_ERR_BOUNDS = -11         /* a kernel computed an index outside its array (only the
                                   bounds-checked build, compiled with RP_CHECKED, tests
                                   this); the access was skipped, results incomplete */
};

/* Where an input array lives. */
enum { RP_MEM_HOST = 0, RP_MEM_DEVICE = 1 };

/* rp_trace_params.flags */
enum {
    RP_FLAG_RAY_HASH = 1,      /* write one 64-bit FNV-1a hash of each primary ray's
                                  triangle sequence (debug/divergence checks) */
    RP_FLAG_COUNT_VISITS = 2,  /* count BVH node visits and triangle tests in stats */
    RP_FLAG_DEVICE_POSITIONS = 4, /* listener and sources are device pointers */
    RP_FLAG_FP32_PATHS = 8,      /* carry path origin, direction and length in FP32 instead
                                    of FP64 (faster; paths drift from the FP64 reference
                                    after tens of reflections) */
    RP_FLAG_SHADOW_PACKETS = 16, /* trace shadow rays as warp packets (32 rays from nearby
                                    reflections to one source walk the BVH together) */
    RP_FLAG_SHADOW_LANES = 32    /* trace shadow rays one per lane, each lane taking a new
                                    ray as soon as its own ends.  Neither flag: packets.
                                    Both flags: RP_ERR_INVALID_ARG.  The two modes give the
                                    same answers. */
};

typedef struct rp_ctx rp_ctx;
typedef struct rp_scene rp_scene;

/* Scene mesh with frequency-dependent materials (Section 5 uses 4 bands).
 * Surfaces are two-sided; triangle winding is not used.  All five arrays are in
 * the memory named by `memory`; they are copied, the caller keeps ownership. */
typedef struct {
    const float *verts;          /* [num_verts][3] metres */
    const int32_t *tris;         /* [num_tris][3] vertex indices */
    const int32_t *tri_material; /* [num_tris] material index */
    const float *absorption;     /* [num_materials][num_bands] alpha in [0,1] */
    const float *scattering;     /* [num_materials][num_bands] s in [0,1] */
    int32_t num_verts;
    int32_t num_tris;
    int32_t num_materials;
    int32_t num_bands;           /* B, 1..RP_MAX_BANDS */
    int32_t memory;              /* RP_MEM_HOST or RP_MEM_DEVICE */
    float ray_epsilon;           /* self-intersection guard t_min; 0 = 1e-6 x bbox diagonal */
} rp_mesh_desc;

typedef struct {
    int32_t num_tris;
    int32_t num_nodes;     /* internal BVH nodes */
    int32_t max_depth;     /* deepest leaf */
    int32_t num_bands;
    float bounds_lo[3];
    float bounds_hi[3];
    float ray_epsilon;     /* t_min used by every ray */
    float build_ms;        /* device time of the BVH build */
    float refit_ms;        /* device time of the last rp_scene_refit's refit launch (0: none) */
} rp_scene_info;

/* One trace step (Section 5): num_rays primaries from the listener, each followed to
 * max_order reflections.  At every reflection of order >= min_order a shadow ray to
 * each source adds the diffusely reflected direct energy; after a specular
 * continuation the next segment also tests the sources as spheres of radius
 * source_radius.  Contributions land in bin floor(t * ir_rate_hz), t = path length / c.
 * Random numbers: Philox4x32-10, counter (ray id, scene_id, bounce, 0), key = seed. */
typedef struct {
    uint64_t num_rays;        /* N primaries (first wave) */
    uint64_t seed;            /* Philox key (lo, hi words) */
    uint64_t first_ray;       /* id of the first primary: rays first_ray .. first_ray + N - 1
                                 (a shard of a larger ray budget); 0 normally */
    int32_t max_order;        /* M reflections per path, >= 0 */
    int32_t sh_order;         /* n, 0..RP_MAX_SH_ORDER */
    int32_t num_bins;         /* T histogram bins, >= 1 */
    int32_t min_order;        /* reflections of lower order are not binned; 0 bins direct sound */
    float ir_rate_hz;         /* IR sample rate (the paper uses 100 Hz) */
    float speed_of_sound;     /* c, m/s */
    float source_radius;      /* r_s, m, > 0 */
    uint32_t scene_id;        /* Philox counter word 1 */
    int32_t budget_refill;    /* 1: spend the unused part of the N*M segment budget on
                                 extra primaries, in deterministic waves (Section 5);
                                 their ray ids follow the first wave's, so
                                 first_ray + N*M <= 2^32.  rp_trace synchronises the
                                 stream while it sizes the waves (N*M <= 2^28: passes
                                 over candidate rays that keep what they trace, the
                                 candidates past the waves dropped; larger budgets:
                                 waves checked every 16), so such a call cannot be
                                 captured into a CUDA graph */
    int32_t flags;            /* RP_FLAG_* */
} rp_trace_params;

/* Direct sound of one source (Section 5, reduced to a point source): visible when the
 * listener-source segment is unoccluded; energy 1/(4 pi d^2) per unit source power in
 * every band, arrival d/c, SH of the direction toward the source times the energy. */
typedef struct {
    int32_t visible;
    int32_t bin;          /* floor(time * ir_rate_hz) */
    float dist;
    float time;
    float energy;
    float sh[RP_MAX_SH];  /* energy * Y_k(direction), k < K */
} rp_direct;

/* Tracer statistics (totals over the whole step, un-normalised unless stated). */
typedef struct {
    double escaped[RP_MAX_BANDS];    /* path weight leaving the scene */
    double absorbed[RP_MAX_BANDS];   /* path weight absorbed by surfaces */
    double remaining[RP_MAX_BANDS];  /* path weight alive after max_order reflections */
    double late[RP_MAX_BANDS];       /* binned energy that fell beyond the last bin,
                                        normalised like H */
    double mfp_sum;                  /* lengths of segments that ended on a surface */
    double mfp_sum_np;               /* the same without primary segments */
    uint64_t mfp_count;
    uint64_t mfp_count_np;
    uint64_t segments;               /* closest-hit rays traced (the segment budget) */
    uint64_t shadow_rays;            /* next-event (diffuse rain) shadow rays traced */
    uint64_t primaries;              /* K primaries over all waves; H is divided by K */
    uint64_t contributions;          /* shadow + sphere contributions (binned or late) */
    uint64_t sphere_hits;
    uint64_t waves;
    uint64_t node_visits[2];         /* with RP_FLAG_COUNT_VISITS: BVH nodes visited by
                                        [0] closest-hit segments, [1] shadow rays */
    uint64_t tri_tests[2];           /* with RP_FLAG_COUNT_VISITS: triangle tests, same split */
    uint64_t hits_stored;            /* reflections kept for next-event estimation */
    uint64_t fp64_reruns;            /* queries whose FP32 answer was rounding-sensitive and
                                        were decided again in FP64 */
    uint64_t packet_walks;           /* with RP_FLAG_COUNT_VISITS: BVH walks of shadow-ray
                                        warp packets (one per packet and job) */
    uint64_t packet_steps;           /* with RP_FLAG_COUNT_VISITS: nodes those walks fetched */
    int32_t error;                   /* first RP_ERR_* raised by a kernel, or 0 */
    int32_t reserved;
} rp_trace_stats;

typedef struct {
    double ir_rate_hz;   /* rate of the histogram */
    double dt_update;    /* seconds since the previous update (smoothing) */
    double tau;          /* smoothing time constant tau, s (paper: 3 s for late reverb);
                            0 disables smoothing */
} rp_estimate_params;

/* Reverberation parameters of one (source, band), Section 4.2. */
typedef struct {
    double rt60_raw;        /* -60 / slope of the least-squares fit; NaN without a fit */
    double rt60_smoothed;   /* exponential smoothing with alpha = 1 - exp(-dt/tau) */
    double fit_hi_db;       /* fit window upper level (-5, -5 or 0 dB) */
    double fit_lo_db;       /* fit window lower level (-35, -25 or -10 dB) */
    double fit_r2;
    double slope_db_per_s;
    double intercept_db;
    double i_total;         /* sum over bins of I(t) */
    double g_reverb;        /* sqrt(i_total / (rt60 / (6 ln 10))) */
    double e_direct;        /* direct energy of the source */
    double drr_db;          /* 10 log10(e_direct / i_total) */
    double predelay_s;      /* first bin non-zero in any band / rate */
    int32_t range_kind;     /* 0 none, 1 T30 (-5..-35 dB), 2 T20 (-5..-25), 3 T10 (0..-10) */
    int32_t n_fit;
    int32_t fit_j0;
    int32_t fit_j1;
    double xbar[RP_MAX_SH]; /* sum_t X_lm(t) / sum_t I(t), k < K */
} rp_reverb_params;

/* Per-kernel device time collected while profiling is enabled. */
typedef struct {
    char name[32];
    uint64_t launches;
    double total_ms;
} rp_kernel_time;

const char *rp_status_string(int status);

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out is owned by the caller
 * until rp_destroy.  Fails with RP_ERR_NO_DEVICE when the device is absent. */
int rp_create(rp_ctx **out, int device, void *cuda_stream);
int rp_destroy(rp_ctx *ctx);
int rp_set_stream(rp_ctx *ctx, void *cuda_stream);

/* Copy the mesh to the device and build its BVH (Morton codes, radix sort,
 * clustering of mutual nearest neighbours in Morton order, all on the device).
 * Non-finite vertices or
 * materials give RP_ERR_NAN_INPUT, zero triangles RP_ERR_EMPTY_SCENE, an index out
 * of range RP_ERR_INVALID_ARG.  Synchronises the stream before returning. */
int rp_scene_create(rp_ctx *ctx, const rp_mesh_desc *mesh, rp_scene **out);
int rp_scene_destroy(rp_scene *scene);

/* Dynamic scenes (Section 6: the benchmark scenes have moving objects; the method is
 * built for interactive propagation in dynamic scenes): new positions for the
 * vertices of an existing scene -- same triangles, materials and vertex count.
 * verts [num_verts][3] metres in the memory named by `memory`, copied.  The BVH keeps
 * its tree and every box is recomputed bottom-up on the device (one launch); the
 * scene bounds, the box padding and the self-intersection guard t_min (when the mesh
 * gave ray_epsilon = 0) are derived from the new positions as a build derives them,
 * so every query answers as it would on a scene built from the moved mesh (the tree
 * decides only the speed).  Large motions make sibling boxes overlap and traversal
 * slower: rebuild with rp_scene_create then.  Non-finite vertices give
 * RP_ERR_NAN_INPUT and leave the scene unchanged; a wrong vertex count gives
 * RP_ERR_INVALID_ARG.  Synchronises the context stream. */
int rp_scene_refit(rp_scene *scene, const float *verts, int32_t num_verts, int32_t memory);
int rp_scene_info_get(const rp_scene *scene, rp_scene_info *out);

/* Reserve the workspace one rp_trace of these sizes needs, so that later calls
 * (and CUDA graph capture of them) allocate nothing. */
int rp_trace_reserve(rp_scene *scene, const rp_trace_params *params, int32_t num_sources);

/* One trace step.
 *   listener  float[3], sources float[num_sources][3]: host memory, or device memory
 *             with RP_FLAG_DEVICE_POSITIONS.
 *   H         device float[S][B][K][T], overwritten: X_{b,k}(t) per source, with
 *             I_b(t) = sqrt(4 pi) * H[s][b][0][t]; normalised per primary ray.
 *   direct    device rp_direct[S] or NULL.
 *   stats     device rp_trace_stats or NULL (zeroed and filled).
 *   ray_hash  device uint64[num_rays] or NULL (with RP_FLAG_RAY_HASH): hashes of
 *             primaries of the first wave.
 * Allocates workspace on first use for these sizes (see rp_trace_reserve). */
int rp_trace(rp_scene *scene, const rp_trace_params *params, const float *listener,
             const float *sources, int32_t num_sources, float *H, rp_direct *direct,
             rp_trace_stats *stats, uint64_t *ray_hash);

/* Estimate reverb parameters from device H [S][B][K][T] (K = (n+1)^2).
 *   direct  device rp_direct[S] or NULL (then e_direct = 0).
 *   out     device rp_reverb_params[S][B].
 *   state   device double[S][B] smoothing state or NULL; NaN entries mean "no
 *           previous value".  Updated in place. */
int rp_estimate(rp_ctx *ctx, const float *H, const rp_direct *direct, int32_t num_sources,
                int32_t num_bands, int32_t num_sh, int32_t num_bins,
                const rp_estimate_params *params, rp_reverb_params *out, double *state);

/* Trace + estimate with HOST buffers: positions are copied in, H, parameters, direct
 * sound and stats are copied out (any output pointer may be NULL).  state is a host
 * double[S][B] or NULL.  Returns after the results are in host memory. */
int rp_update(rp_scene *scene, const rp_trace_params *params,
              const rp_estimate_params *est, const float *listener, const float *sources,
              int32_t num_sources, float *H_host, rp_reverb_params *params_host,
              rp_direct *direct_host, rp_trace_stats *stats_host, double *state_host);

/* ---------------------------------------------------------------------------
 * Reverberator parameters (Section 4.1 "Sound Rendering", Section 4.2 "Reflection
 * Density"): the SH-domain Schroeder reverberator of each source has RP_N_COMB comb
 * filters in parallel (then all-pass filters in series).
 * --------------------------------------------------------------------------- */
#define RP_N_COMB 8

typedef struct {
    double mean_delay_s;      /* r_free / c the comb delays were drawn for (state) */
    uint32_t generation;      /* draws so far (state; 0 before the first: zero the struct) */
    int32_t resampled;        /* 1 when this update drew new delays */
    double t_comb[RP_N_COMB];                     /* feedback delays, s */
    double g_comb[RP_N_COMB][RP_MAX_BANDS];       /* feedback gains 10^(-3 t_comb / RT60_b) (0: no RT60) */
    double dir[RP_N_COMB][3];                     /* dominant direction of each comb's input */
    float comb_in[RP_N_COMB][RP_MAX_SH];          /* input SH gains Y_lm(dir) / RP_N_COMB */
    float rot[RP_N_COMB][3][3];                   /* the comb's rotation Rz(g) Ry(b) Rx(a) */
    float J[RP_N_COMB][RP_MAX_SH][RP_MAX_SH];     /* its SH rotation: Y(rot d) = J Y(d) */
    float D[RP_MAX_BANDS][RP_MAX_SH][RP_MAX_SH];  /* directional loudness per band */
} rp_reverberator;

/* The reverberator parameters of S sources from their IR H [S][B][K][T] and
 * rp_estimate's parameters [S][B] (smoothed RT60, average directivity xbar), device
 * memory; rev: device rp_reverberator[S], zeroed before the first update, updated in
 * place (the comb delays persist between updates):
 *   comb delays: N(r_free / c, sigma = (r_free / c) / 3) per comb (Section 4.2), at
 *     least a tenth of the mean, drawn from Philox (key seed, counter (source, comb,
 *     generation, 3)) by Box-Muller, and drawn again only when r_free / c moved by
 *     more than 2 sigma from the mean of the last draw;
 *   comb gains: 10^(-3 t_comb / RT60_b) (comb feedback gain equation);
 *   comb input: the dominant direction normalize(-X_11, -X_1-1, X_10) of the
 *     band-summed first-order IR at t_comb past its first non-zero bin (linear
 *     interpolation; +z when it vanishes), and Y_lm(dir) / N_comb (Section 4.1);
 *   rotations: per comb a random rotation, angles uniform in [90, 270] degrees about
 *     x, y and z (Philox counter (source, comb, 0, 2)), and its SH rotation matrix by
 *     the recurrence of Ivanic and Ruedenberg (Section 4.1 "SH Rotations");
 *   directional loudness: D_b = sum_j w_j a(x_j) Y(x_j) Y(x_j)^T over a product Gauss
 *     rule of the sphere (2n + 2 Gauss-Legendre nodes in cos(theta) x 4n + 4
 *     azimuths, standing in for the paper's spherical t-design), a(x) the amplitude
 *     gain sqrt(max(f(x), 0) / mean f) of the average directivity's density
 *     f(x) = sum_k xbar_k Y_k(x); the identity for isotropic reverberation.
 * mean_free_path: rp_trace_stats' mfp_sum / mfp_count (m). */
int rp_reverb_configure(rp_ctx *ctx, const float *H, const rp_reverb_params *params, int32_t num_sources,
                        int32_t num_bands, int32_t num_sh, int32_t num_bins, double ir_rate_hz,
                        double mean_free_path, double speed_of_sound, uint64_t seed, rp_reverberator *rev);

/* The reverberator itself (Section 4.1 "Sound Rendering"; Section 5 "Auralization"),
 * rendered for many sources at once, block by block:
 *   bands     a serial Linkwitz-Riley 4th-order crossover (2nd-order Butterworth
 *             biquads applied twice, bilinear transform, FP64 state): band 0 is the
 *             low part at crossover_hz[0], the high part is split again at the next
 *             frequency, band B-1 is the last high part;
 *   predelay  each band read round(predelay_s x fs) samples late (rp_reverb_params);
 *   combs     RP_N_COMB in parallel in the SH domain: y[n] = comb_in x[n - p] +
 *             g_comb J y[n - d], d = max(1, round(t_comb fs)) -- every pass through
 *             the feedback rotates the delayed K-vector by the comb's J and scales it;
 *   all-pass  4 in series per (band, SH channel): v[n] = -0.7 u[n] + u[n - d] +
 *             0.7 v[n - d], d = 5, 1.7, 0.6, 0.2 ms (the paper gives only the count);
 *   output    q[n] = sum_b g_reverb_b D_b v_b[n]: K SH channels per source.
 * Comb delays above max_delay_samples or a predelay above max_predelay_samples are
 * clamped and RP_ERR_CAPACITY is recorded. */
typedef struct {
    double sample_rate;                        /* fs, Hz */
    double crossover_hz[RP_MAX_BANDS - 1];     /* B - 1 increasing frequencies below fs / 2
                                                  (the paper's 4 bands: 176, 775, 3408 Hz) */
    int32_t max_delay_samples;                 /* comb ring length */
    int32_t max_predelay_samples;
} rp_reverb_render_config;

/* Bytes of the render state of S sources (device memory the caller owns; zero it
 * before the first block -- the rings, crossover states and sample counters). */
int rp_reverb_state_bytes(int32_t num_sources, int32_t num_bands, int32_t num_sh, const rp_reverb_render_config *cfg,
                          int64_t *bytes);
/* One block of N samples: in [S][N] (device, mono source signals), out [S][K][N]
 * (device); rev [S] (rp_reverb_configure) and params [S][B] (rp_estimate) device
 * memory; state as rp_reverb_state_bytes says, carried from block to block. */
int rp_reverb_render(rp_ctx *ctx, const rp_reverberator *rev, const rp_reverb_params *params, int32_t num_sources,
                     int32_t num_bands, int32_t num_sh, const rp_reverb_render_config *cfg, const float *in,
                     int32_t num_samples, float *out, void *state);

/* ---------------------------------------------------------------------------
 * Temporal coherence (Section 5, "Sound Propagation"): the early reflections (the
 * first orders; the paper uses 2) go to a diffuse path cache with spherical-harmonic
 * directivity per path, smoothed over updates (tau_ER = 1 s in the paper); the N_ER
 * most intense early paths (100 among all sources) are rendered and the others are
 * added to the late IR before it is analysed; the late IR itself is smoothed by an
 * impulse response cache (tau_LR = 3 s).
 * --------------------------------------------------------------------------- */
typedef struct rp_er_cache rp_er_cache;

/* One early path: the diffuse-rain contributions of this cache's source through the
 * same reflections, summed (reading of the paper's diffuse path cache):
 * energy[b] = sum of e_b / K, sh[b][k] = sum of e_b Y_k(d0) / K (d0: each
 * contribution's arrival direction, its path's first segment), delay = the
 * energy-weighted mean arrival time; K = primaries of the update. */
typedef struct {
    int32_t source;
    int32_t order;                          /* 1 or 2 */
    int32_t tri[2];                         /* input triangle of reflections 1 and 2 (-1: none) */
    double delay_s;
    double energy[RP_MAX_BANDS];            /* per unit source power, b < B */
    double sh[RP_MAX_BANDS][RP_MAX_SH];     /* b < B, k < K */
} rp_er_path;

typedef struct {
    double dt_update;          /* seconds since the previous update */
    double tau_er;             /* smoothing time constant of the path cache (paper: 1 s); 0: none */
    double prune;              /* cached paths whose total energy falls to this or below are dropped */
    double hearing_threshold;  /* paths whose total energy is at or below this are not rendered
                                  (the listener's threshold of hearing, per unit source power) */
    int32_t n_er;              /* paths rendered per update among all sources (paper: 100) */
    int32_t reserved;
} rp_er_params;

/* A path cache for num_bands bands and SH order sh_order (owned by the caller until
 * rp_er_cache_destroy; its device arrays grow as the cache does). */
int rp_er_cache_create(rp_ctx *ctx, int32_t num_bands, int32_t sh_order, rp_er_cache **out);
int rp_er_cache_destroy(rp_er_cache *cache);
/* Forget every path: the next update starts the cache (alpha = 1). */
int rp_er_cache_reset(rp_er_cache *cache);
/* The cached paths in key order (source, triangle of reflection 1, of reflection 2,
 * an order-1 path after the order-2 paths of its triangle) into device out[max_paths];
 * *count (host) = paths in the cache. */
int rp_er_cache_read(rp_er_cache *cache, rp_er_path *out, int64_t max_paths, int64_t *count);

/* rp_trace with the early reflections kept apart (2 <= min_order <= 3: orders below
 * min_order are early; at most 2):
 *   1. the trace step as rp_trace: H holds orders >= min_order;
 *   2. every early reflection's diffuse-rain shadow ray to every source; each visible
 *      one is a contribution of the path (source, its reflections' triangles);
 *   3. this update's paths, updated into the cache: energy and SH as
 *      (1 - alpha) cached + alpha new, alpha = 1 - exp(-dt_update / tau_er) (1 on the
 *      cache's first update), delay weighted by energy; paths pruned as ep->prune says;
 *   4. the cached paths above the hearing threshold sorted by decreasing total energy
 *      (ties in key order): the first n_er are written to `rendered` (device
 *      rp_er_path[n_er]), their number to *num_rendered (device int32); the others are
 *      added to H at bin floor(delay x ir_rate_hz) (dropped past the last bin).
 * The cache's band count and SH order must match the scene and params; the scene
 * must have fewer than 2^21 - 1 triangles and S < 4096.  Synchronises the stream
 * (sizes are read back between the steps). */
int rp_trace_er(rp_scene *scene, const rp_trace_params *params, const float *listener, const float *sources,
                int32_t num_sources, float *H, rp_direct *direct, rp_trace_stats *stats, rp_er_cache *cache,
                const rp_er_params *er, rp_er_path *rendered, int32_t *num_rendered);

/* The impulse response cache of the late IR: C = (1 - alpha) C + alpha H over `count`
 * cells (device float arrays), alpha = 1 - exp(-dt_update / tau) (paper: tau_LR =
 * 3 s), or C = H when `first` is nonzero or tau = 0.  rp_estimate then runs on C. */
int rp_ir_cache_update(rp_ctx *ctx, const float *H, float *C, int64_t count, double dt_update, double tau,
                       int32_t first);

/* ---------------------------------------------------------------------------
 * Batched updates: many independent scenes, each with its own sources, listener and
 * ray budget, traced in the same persistent launches and estimated together; the
 * whole update can be captured once in a CUDA graph and replayed per update.
 * --------------------------------------------------------------------------- */
typedef struct rp_batch rp_batch;

typedef struct {
    rp_scene *scene;        /* created on the batch's context; same band count for all items */
    const float *listener;  /* host float[3] */
    const float *sources;   /* host float[num_sources][3] */
    int32_t num_sources;
    uint32_t scene_id;      /* Philox counter word 1 of this item */
    uint64_t num_rays;
    uint64_t first_ray;
} rp_batch_item;

/* Launch shape of a batch, chosen by rp_batch_autotune or set by hand. */
typedef struct {
    int32_t chunk_rays;            /* primaries per work chunk of the paths kernel, 32..65536 */
    int32_t shadow_steps;          /* BVH nodes a shadow-ray lane visits between refills, 1..64 */
    int32_t paths_blocks_per_sm;   /* persistent grid of the paths kernel, 1..occupancy */
    int32_t shadow_blocks_per_sm;  /* persistent grid of the shadow-ray kernel, 1..occupancy */
    int32_t shadow_mode;           /* 0: the default (packets, see RP_FLAG_SHADOW_LANES),
                                      1: packets, 2: one ray per lane */
} rp_batch_tuning;

typedef struct {
    int32_t num_items;
    int32_t total_sources;
    int32_t num_groups;                  /* steps the update is split into (memory budget) */
    int32_t reserved;
    uint64_t total_rays;
    uint64_t max_group_reflections;
} rp_batch_info;

/* Create a batch of num_items items sharing `params` (max_order, sh_order, num_bins,
 * min_order, ir_rate_hz, speed_of_sound, source_radius, flags; num_rays, first_ray,
 * scene_id and seed are per item / per run; budget_refill, RP_FLAG_RAY_HASH and
 * RP_FLAG_DEVICE_POSITIONS are rejected).  Item i's sources take global indices
 * sum_{i'<i} num_sources(i') ... in the outputs, all device memory owned by the caller:
 *   H       float[total sources][B][K][T], each item normalised by its own primaries
 *   direct  rp_direct[total sources]
 *   params  rp_reverb_params[total sources][B] or NULL (no estimation); est must be set
 *   stats   rp_trace_stats (aggregate over the batch) or NULL
 * Positions are copied at creation.  Workspace is reserved here; later calls on the
 * context that grow it make the next graph run re-capture.  Items are traced in
 * groups whose stored reflections fit 2^27 slots (about 11 GB at 8 bands); the
 * environment variable RP_BATCH_HIT_BUDGET can lower that budget. */
int rp_batch_create(rp_ctx *ctx, const rp_batch_item *items, int32_t num_items,
                    const rp_trace_params *params, const rp_estimate_params *est, float *H,
                    rp_direct *direct, rp_reverb_params *params_out, rp_trace_stats *stats,
                    rp_batch **out);
int rp_batch_destroy(rp_batch *batch);

/* Enqueue one batched update with Philox key `seed`.  use_graph = 1 captures the
 * launch sequence into a CUDA graph on first use (or after a tuning or workspace
 * change) and replays it; the key is read from device memory, so replays take new
 * keys.  Asynchronous: rp_sync_status(ctx) waits and reports device errors. */
int rp_batch_run(rp_batch *batch, uint64_t seed, int use_graph);

int rp_batch_set_tuning(rp_batch *batch, const rp_batch_tuning *tuning);
int rp_batch_get_tuning(const rp_batch *batch, rp_batch_tuning *tuning);
int rp_batch_info_get(const rp_batch *batch, rp_batch_info *out);

/* Time launch shapes on this batch (coordinate descent over the shadow-ray mode
 * {packets, lanes}, shadow_steps {4,8,16}, chunk_rays {64,256,1024} and full or half
 * persistent grids, two runs each) and apply the fastest.  cache_path (or NULL) is a
 * text file of "key chunk steps paths_blocks shadow_blocks mode ms" lines keyed by
 * device, SM count and batch shape; a cached entry is applied without timing. */
int rp_batch_autotune(rp_batch *batch, uint64_t seed, const char *cache_path,
                      rp_batch_tuning *best, double *best_ms);

/* ---------------------------------------------------------------------------
 * Learned estimator: an MLP that maps the energy IR of a low-ray-count trace plus
 * scene features to per-band decay times and direct-to-reverberant ratios, trained
 * on IRs the method itself produces at high ray counts.  BF16 tensor-core GEMMs with
 * FP32 accumulation, FP32 master weights, AdamW (beta1 0.9, beta2 0.999, eps 1e-8).
 * The paper has no learned part; the plain estimator (rp_estimate) stays the
 * reference the network is judged against.  All arrays are device memory unless
 * stated otherwise.
 * --------------------------------------------------------------------------- */
typedef struct rp_mlp rp_mlp;

enum { RP_MLP_FLAG_LEGACY_GEMM = 1 /* every GEMM on the mma.sync kernels (for comparison) */ };

typedef struct {
    int32_t in_dim;     /* input features, >= 522 and a multiple of 8 (features below) */
    int32_t hidden;     /* width of each hidden layer, multiple of 8 */
    int32_t layers;     /* hidden layers (GELU), 1..8 */
    int32_t out_dim;    /* outputs (16: log RT60 [s] and DRR [dB] per band) */
    int32_t max_batch;  /* largest n of one call */
    int32_t flags;      /* RP_MLP_FLAG_*; 0: the forward pass runs as one fused tcgen05
                           tensor-core launch (TMA-staged operands, TMEM accumulators)
                           when hidden is a multiple of 64 up to 256, out_dim a multiple of
                           16 up to 256 and layers <= 8, else on mma.sync GEMMs; the
                           backward pass runs on mma.sync GEMMs */
    uint64_t seed;      /* weight initialisation: uniform +-sqrt(6/(in+out)) from Philox */
} rp_mlp_config;

/* Scene features of a scene, host float[10]: log10 of the bounding-box volume,
 * log10 of the total triangle area, area-weighted mean absorption of bands 0..7
 * (0 beyond the scene's band count). */
int rp_scene_features(rp_scene *scene, float *out);

/* Raw features X[S][in_dim] (float) of the S sources of H[S][B][K][T] (B <= 8,
 * 4 <= T <= 11264).  Per band b: the energy-decay (Schroeder) curve of the band's
 * omnidirectional series, D(t) = sum over t' >= t of H[s][b][0][t'], divided by D(0);
 * t_end = the first bin where it is below 1e-4 (-40 dB; T when it never is; at least
 * 4); X[b*64 + i] = log10(D(t_end * (i+1) / 63) + 1e-8) for i = 0..62, D taken
 * between bins by linear interpolation (positions clamped to T - 1.001), and
 * X[b*64 + 63] = ln(t_end / ir_rate_hz).  An empty band (or b >= B) gives -8 and
 * ln(4 / ir_rate_hz).  Then scene_feats[S][10] (rp_scene_features) at 512..521 and
 * zeros up to in_dim.  The decay curve is the backward energy integral that the
 * plain estimator fits (Section 4.2, "Reverberation Time"); the window makes the
 * features scale-free in time.
 * RP_ERR_TOO_LARGE when T > 11264. */
int rp_mlp_features(rp_ctx *ctx, const float *H, int32_t num_sources, int32_t num_bands,
                    int32_t num_sh, int32_t num_bins, float ir_rate_hz, const float *scene_feats,
                    int32_t in_dim, float *X);

int rp_mlp_create(rp_ctx *ctx, const rp_mlp_config *config, rp_mlp **out);
int rp_mlp_destroy(rp_mlp *mlp);
int rp_mlp_param_count(const rp_mlp *mlp, int64_t *count);
/* FP32 master parameters, layer by layer W[in][out] then b[out]; set refreshes the
 * BF16 copies.  Together with the AdamW state they are a training checkpoint. */
int rp_mlp_get_params(rp_mlp *mlp, float *params);
int rp_mlp_set_params(rp_mlp *mlp, const float *params);
int rp_mlp_get_adam_state(rp_mlp *mlp, float *m, float *v, int32_t *step);
int rp_mlp_set_adam_state(rp_mlp *mlp, const float *m, const float *v, int32_t step);
/* Standardisation of inputs and targets (host arrays): x' = (x - mean) / std, y = y' std + mean. */
int rp_mlp_set_normalization(rp_mlp *mlp, const float *in_mean, const float *in_std,
                             const float *out_mean, const float *out_std);
/* Standardise raw features X[n][in_dim] into the BF16 network input Xb[n][in_dim]. */
int rp_mlp_prepare(rp_mlp *mlp, const float *X, int32_t n, void *Xb);
/* Y[n][out_dim] = network(Xb), de-standardised when destandardize != 0. */
int rp_mlp_forward(rp_mlp *mlp, const void *Xb, int32_t n, float *Y, int32_t destandardize);
/* Masked MSE on standardised targets T[n][out_dim] with mask[n][out_dim] (0 or 1):
 * loss = sum mask (y - t)^2 / max(1, sum mask); loss (device float) and the gradient
 * in the parameter layout (or NULL). */
int rp_mlp_loss_grad(rp_mlp *mlp, const void *Xb, const float *T, const float *mask, int32_t n,
                     float *loss, float *grad);
/* One AdamW step on that loss (decoupled weight decay). loss may be NULL. */
int rp_mlp_train_step(rp_mlp *mlp, const void *Xb, const float *T, const float *mask, int32_t n,
                      float lr, float weight_decay, float *loss);

/* Size of the fixed device scratch array used by rp_trace_noalloc: 64 MiB, held by
 * every GPU that loads the library for the life of the process. */
#define RP_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* rp_trace without any memory allocation.  The paper has no counterpart: it exists
 * for callers that must not allocate device memory during an update -- a real-time
 * audio or game thread that cannot block on the driver's allocator mid-frame, or an
 * application that hands out all device memory from its own pool and does not let
 * libraries allocate.  Same arguments and outputs as rp_trace (no ray hashes); the
 * scene and context are created beforehand with rp_create / rp_scene_create.  All
 * temporaries come from one static __device__ array of RP_NOALLOC_SCRATCH_BYTES; no
 * cudaMalloc, cudaFree or other allocating call is made.
 * Size limit: the problem fits when, with R = num_rays x max_order (stored
 * reflections, worst case) and B bands, these together stay within the array:
 *   (96 + 8 B) bytes per reflection (stored reflections, their spatial order and the
 *   cell-ordered copy the shadow rays read), 1 MiB of cell counts, 12 B per (source,
 *   bin) (counting sort), 8 B per histogram cell S x B x K x T (compensated sums),
 *   and room for at least R / 2 + 4096 + S contribution records of
 *   (29 + 4 B + ceil((8 + 16 B K) / 1024)) bytes each (key, ray id, energies, sort
 *   index and the shares of the FP64 re-decision queue and of the segment sums of
 *   heavy (source, bin) keys).  Larger problems return RP_ERR_TOO_LARGE before any
 *   work is enqueued.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current): make that first call before any stream capture begins.
 * Every call shares the array and
 * overwrites the previous call's temporaries, so calls that may overlap on the GPU
 * (several streams or host threads) race and must be serialised by the caller.
 * Host positions are copied with cudaMemcpyAsync, and budget_refill reads the waves'
 * sizes back (the stream is synchronised), as in rp_trace. */
int rp_trace_noalloc(rp_scene *scene, const rp_trace_params *params, const float *listener,
                     const float *sources, int32_t num_sources, float *H, rp_direct *direct,
                     rp_trace_stats *stats);

/* Limits for exercising the error paths without faulting the GPU (the paper has no
 * counterpart).  All zero means the normal limits.  rp_trace and rp_update of the
 * context apply them until they are reset:
 *   iter_cap    node visits of one BVH traversal query (closest hit, shadow ray or
 *               direct sound) before it stops and records RP_ERR_TIMEOUT; normally
 *               4 x internal nodes + 64, which a query of a well-formed tree never
 *               reaches.  A query stopped this way answers with what it found so far.
 *   hit_cap     stored-reflection slots of a trace step; normally num_rays x max_order
 *               (the worst case).  Reflections past it are dropped and RP_ERR_CAPACITY
 *               is recorded.
 *   record_cap  contribution records held at once; normally the worst case of a record
 *               chunk.  Records past it are dropped and RP_ERR_CAPACITY is recorded.
 *   spec_slots  the budget refill's planner (budget_refill): speculative candidates a
 *               store pass keeps apart; normally max(4 N, 8192).  A store pass traces
 *               candidate rays once and keeps their results; with too few slots it
 *               gives up and the planned rays are traced again (the same results).
 *               -1: no store passes (counting passes, then the planned rays).  A
 *               nonzero hit_cap or record_cap also turns the store passes off.
 * The errors come back from rp_sync_status (and in rp_trace_stats.error); the context
 * stays usable, and the next call after the limits are reset runs normally.
 * limits = NULL resets them. */
typedef struct {
    int32_t iter_cap;
    int32_t spec_slots;
    uint64_t hit_cap;
    uint64_t record_cap;
} rp_debug_limits;
int rp_set_debug_limits(rp_ctx *ctx, const rp_debug_limits *limits);

/* Measured throughput of the FP32 pipes that bound BVH traversal (a calibration for
 * rooflines; the paper has no counterpart): *fma_per_s = FP32 fused multiply-add
 * instructions per second (2 flops each), *minmax_per_s = FP32 min/max instructions
 * per second, each from independent chains filling every SM, timed with CUDA events
 * on the context stream (best of five).  Allocates a small buffer and synchronises. */
int rp_measure_pipe_peaks(rp_ctx *ctx, double *fma_per_s, double *minmax_per_s);

/* Synchronise the context stream and return the first device-side error (or a CUDA
 * error).  Clears the recorded device error. */
int rp_sync_status(rp_ctx *ctx);

/* Kernel timing with CUDA events on the context stream (off by default). */
int rp_profile_enable(rp_ctx *ctx, int enable);
int rp_profile_reset(rp_ctx *ctx);
int rp_profile_read(rp_ctx *ctx, rp_kernel_time *out, int32_t max_entries, int32_t *count);

#ifdef __cplusplus
}
#endif

#endif /* RPR_H */
