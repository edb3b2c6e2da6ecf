// coherence.cu -- temporal coherence of Section 5: the early-reflection diffuse path
// cache with spherical-harmonic directivity per path, the prioritisation of early
// paths (the N_ER most intense are rendered, the others join the late IR before it is
// analysed), and the impulse-response cache that smooths the late IR over updates.
//
// One rp_trace_er update:
//   1. the trace step (trace.cu) with early reflections -- orders 1 .. min_order - 1,
//      at most 2 -- kept apart by k_paths;
//   2. k_er_shadow: the diffuse-rain shadow ray of every early reflection to every
//      source; a visible one is a record keyed by (source, original triangle of
//      reflection 1, of reflection 2 or none), with its energy per band, path length
//      (FP64 positions) and primary ray;
//   3. a stable LSD radix sort of the records by key; one warp per key reduces its
//      records to this update's path: energy per band and SH directivity divided by
//      the primaries, delay = energy-weighted mean arrival time (FP64 sums);
//   4. merge with the cache (both sorted by key; merge positions by binary search):
//      every key keeps (1 - alpha) cached + alpha new, the delay weighted by energy;
//      paths whose total energy falls to the prune level are dropped;
//   5. prioritisation: a stable sort by decreasing total energy (equal energies in key
//      order); paths above the hearing threshold are rendered up to N_ER, the rest of
//      them are added to H at floor(delay x rate) with their SH energy.
#include <cmath>
#include <new>

#include "handles.cuh"
#include "traverse.cuh"

using namespace rp;

namespace rp {
namespace {

constexpr int ER_THREADS = 128;
constexpr unsigned long long ER_TRI_BITS = 21;
constexpr unsigned long long ER_TRI_NONE = (1ull << ER_TRI_BITS) - 1;  // no reflection 2 (order-1 path)
constexpr int RS_WORKERS_MAX = 2048;

__device__ __forceinline__ unsigned long long er_key(int s, unsigned t1, unsigned t2)
{
    return ((unsigned long long)s << (2 * ER_TRI_BITS)) | ((unsigned long long)t1 << ER_TRI_BITS) | t2;
}

// 2. shadow rays of the early reflections; item q = (reflection q / S, source q % S)
__global__ void __launch_bounds__(ER_THREADS) k_er_shadow(TraceWork w, unsigned long long *rkey, float *re,
                                                          double *rlen, uint32_t *rrid, unsigned long long cap,
                                                          unsigned long long *count)
{
    __shared__ int sstack[SMEM_STACK * ER_THREADS];
    const unsigned long long n = min(w.ctr->n_er, w.er.cap);
    const int S = w.k.S, B = w.k.B;
    const SceneView &sc = w.job0.sc;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n * S;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long j = q / S;
        const int s = (int)(q - j * S);
        const float4 P = w.er.hits.p[j], N = w.er.hits.n[j], lo = w.er.hits.plo[j];
        const float4 cs = __ldg(w.pos + s);
        const float3 v = xyz(cs) - xyz(P);
        const float dist2 = dot(v, v), dist = sqrtf(dist2);
        const float cth = dot(xyz(N), v) / dist;
        if (!(cth > 0.f)) continue;
        const int tri = __float_as_int(N.w);
        TravStats ts = {0u, 0u};
        float tt;
        bool amb = false;
        const float3 dir = v * (1.0f / dist);
        int blk = traverse<true, false, true>(sc, xyz(P), dir, sc.tmin, dist, tri, sstack + threadIdx.x, tt, ts,
                                              w.status, &amb);
        const D3 pd = {(double)P.x + lo.x, (double)P.y + lo.y, (double)P.z + lo.z};
        const double vx = (double)cs.x - pd.x, vy = (double)cs.y - pd.y, vz = (double)cs.z - pd.z;
        const double dd = sqrt(vx * vx + vy * vy + vz * vz);
        if (amb) {
            double te;
            blk = traverse_exact<true>(sc, pd, D3{vx / dd, vy / dd, vz / dd}, sc.tmin_d, dd, tri,
                                       sstack + threadIdx.x, te, w.status);
        }
        if (blk >= 0) continue;
        const unsigned long long r = atomicAdd(count, 1ull);
        if (r >= cap) {
            raise_error(w.status, RP_ERR_CAPACITY);
            continue;
        }
        // original triangle indices of the path's reflections
        const unsigned t2leaf = (unsigned)tri;
        const int prev = w.er.prev[j];
        const unsigned o_cur = __float_as_uint(__ldg(sc.tris + 3 * t2leaf + 1).w);
        unsigned t1, t2;
        if (prev < 0) {
            t1 = o_cur;
            t2 = (unsigned)ER_TRI_NONE;
        } else {
            t1 = __float_as_uint(__ldg(sc.tris + 3 * prev + 1).w);
            t2 = o_cur;
        }
        rkey[r] = er_key(s, t1, t2);
        const float f = cth * (1.0f / PI_F) / dist2;
        for (int b = 0; b < B; ++b) re[r * B + b] = w.er.hits.ws[j * B + b] * f;
        rlen[r] = (double)P.w + (double)lo.w + dd;
        rrid[r] = w.er.hits.rid[j];
    }
}

// --- stable LSD radix sort of 64-bit keys with 32-bit values (8 bits a pass) -------
// Worker t takes the contiguous slice [t L, (t+1) L) in order; the destinations of
// digit d are the exclusive scan over (d, worker) of the counts, so equal digits keep
// their order.
__global__ void k_rs64_count(const unsigned long long *__restrict__ keys, int n, int shift, int W, int L,
                             uint32_t *__restrict__ counts)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W) return;
    uint32_t c[256];
    for (int d = 0; d < 256; ++d) c[d] = 0u;
    const int a = t * L, b = min(n, a + L);
    for (int i = a; i < b; ++i) c[(keys[i] >> shift) & 255ull]++;
    for (int d = 0; d < 256; ++d) counts[d * W + t] = c[d];
}

__global__ void k_rs64_scatter(const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
                               unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout, int n, int shift,
                               int W, int L, const uint32_t *__restrict__ offs)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W) return;
    uint32_t o[256];
    for (int d = 0; d < 256; ++d) o[d] = offs[d * W + t];
    const int a = t * L, b = min(n, a + L);
    for (int i = a; i < b; ++i) {
        const unsigned long long k = kin[i];
        const uint32_t pos = o[(k >> shift) & 255ull]++;
        kout[pos] = k;
        vout[pos] = vin[i];
    }
}

__global__ void k_iota(uint32_t *v, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

// 3. segment heads of the sorted keys
__global__ void k_heads(const unsigned long long *__restrict__ k, int n, uint32_t *__restrict__ head)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) head[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void k_starts(const uint32_t *__restrict__ head, const uint32_t *__restrict__ pos, int n,
                         uint32_t *__restrict__ start)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && head[i]) start[pos[i]] = (uint32_t)i;
    if (i == 0) start[pos[n]] = (uint32_t)n;  // pos[n] = number of segments
}

// one warp per path: records staged 32 at a time (energy, SH of the primary direction
// from Philox, arrival time), cells summed in FP64 by the lanes that own them
__global__ void __launch_bounds__(128) k_path_reduce(TraceWork w, const unsigned long long *__restrict__ skey,
                                                     const uint32_t *__restrict__ sidx,
                                                     const uint32_t *__restrict__ start, const uint32_t *npaths,
                                                     const float *__restrict__ re, const double *__restrict__ rlen,
                                                     const uint32_t *__restrict__ rrid, unsigned long long *pkey,
                                                     double *pE, double *pX, double *pdelay)
{
    __shared__ float se[4][32][MAXB];
    __shared__ float sy[4][32][MAXK];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int B = w.k.B, K = w.k.K, BK = B * K;
    const unsigned long long seed = w.seed_val;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const double kp = (double)max(w.js[0].primaries, 1ull);
    const double inv_c = 1.0 / (double)w.k.c;
    const int P = (int)*npaths;
    for (int p = blockIdx.x * 4 + wp; p < P; p += gridDim.x * 4) {
        const uint32_t a = start[p], b = start[p + 1];
        double X[4] = {0.0, 0.0, 0.0, 0.0}, E = 0.0, num = 0.0, den = 0.0;
        for (uint32_t base = a; base < b; base += 32) {
            const int cnt = (int)min(32u, b - base);
            double et = 0.0, el = 0.0;
            if (lane < cnt) {
                const uint32_t r = sidx[base + lane];
                float tot = 0.f;
                for (int bb = 0; bb < MAXB; ++bb) {
                    const float v = bb < B ? re[(size_t)r * B + bb] : 0.f;
                    se[wp][lane][bb] = v;
                    tot += v;
                }
                const float3 d0 = primary_direction(rrid[r], w.job0.scene_id, key0, key1);
                float Y[MAXK];
                sh_eval(w.k.sh_order, d0.x, d0.y, d0.z, Y);
                for (int kk = 0; kk < MAXK; ++kk) sy[wp][lane][kk] = kk < K ? Y[kk] : 0.f;
                et = (double)tot;
                el = et * rlen[r] * inv_c;
            }
            __syncwarp();
            for (int i = 0; i < 4; ++i) {
                const int c = lane + 32 * i;
                if (c < BK) {
                    const int bb = c / K, kk = c - bb * K;
                    for (int j = 0; j < cnt; ++j) X[i] += (double)se[wp][j][bb] * (double)sy[wp][j][kk];
                }
            }
            if (lane < B)
                for (int j = 0; j < cnt; ++j) E += (double)se[wp][j][lane];
            for (int o = 16; o > 0; o >>= 1) {
                et += __shfl_xor_sync(FULL, et, o);
                el += __shfl_xor_sync(FULL, el, o);
            }
            den += et;
            num += el;
            __syncwarp();
        }
        for (int i = 0; i < 4; ++i) {
            const int c = lane + 32 * i;
            if (c < BK) pX[(size_t)p * BK + c] = X[i] / kp;
        }
        if (lane < B) pE[(size_t)p * B + lane] = E / kp;
        if (lane == 0) {
            pkey[p] = skey[a];
            pdelay[p] = den > 0.0 ? num / den : 0.0;
        }
    }
}

// --- 4. merge with the cache ------------------------------------------------------
constexpr uint32_t FROM_FRAME = 0x80000000u;

__device__ __forceinline__ int lower_bound64(const unsigned long long *a, int n, unsigned long long k)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (a[m] < k) lo = m + 1;
        else hi = m;
    }
    return lo;
}

__device__ __forceinline__ int upper_bound64(const unsigned long long *a, int n, unsigned long long k)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (a[m] <= k) lo = m + 1;
        else hi = m;
    }
    return lo;
}

__global__ void k_merge_pos(const unsigned long long *ckey, int nc, const unsigned long long *fkey, int nf,
                            unsigned long long *mkey, uint32_t *msrc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) {
        const int pos = i + lower_bound64(fkey, nf, ckey[i]);  // a cached path before a new one of its key
        mkey[pos] = ckey[i];
        msrc[pos] = (uint32_t)i;
    } else if (i < nc + nf) {
        const int j = i - nc;
        const int pos = j + upper_bound64(ckey, nc, fkey[j]);
        mkey[pos] = fkey[j];
        msrc[pos] = (uint32_t)j | FROM_FRAME;
    }
}

struct CacheArrays {
    unsigned long long *key;
    double *E, *X, *delay;
};

// weighted energy of merged entry m (cache entries x (1 - alpha), new ones x alpha)
__device__ __forceinline__ double entry_total(const CacheArrays &c, const CacheArrays &f, uint32_t src, int B,
                                              double alpha)
{
    const bool fr = (src & FROM_FRAME) != 0;
    const uint32_t i = src & ~FROM_FRAME;
    const double *E = fr ? f.E : c.E;
    double t = 0.0;
    for (int b = 0; b < B; ++b) t += E[(size_t)i * B + b];
    return (fr ? alpha : 1.0 - alpha) * t;
}

// keep[m] = 1 for the first entry of a key whose combined energy is above `prune`
__global__ void k_merge_flags(const unsigned long long *mkey, const uint32_t *msrc, int n, CacheArrays c,
                              CacheArrays f, int B, double alpha, double prune, uint32_t *keep)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    uint32_t k = 0u;
    if (m == 0 || mkey[m] != mkey[m - 1]) {
        double t = entry_total(c, f, msrc[m], B, alpha);
        if (m + 1 < n && mkey[m + 1] == mkey[m]) t += entry_total(c, f, msrc[m + 1], B, alpha);
        k = t > prune ? 1u : 0u;
    }
    keep[m] = k;
}

__global__ void k_merge_write(const unsigned long long *mkey, const uint32_t *msrc, int n, const uint32_t *keep,
                              const uint32_t *pos, CacheArrays c, CacheArrays f, int B, int BK, double alpha,
                              CacheArrays out)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n || !keep[m]) return;
    const uint32_t o = pos[m];
    double Et = 0.0, num = 0.0;
    double E[MAXB];
    for (int b = 0; b < MAXB; ++b) E[b] = 0.0;
    const int parts = (m + 1 < n && mkey[m + 1] == mkey[m]) ? 2 : 1;
    for (int q = 0; q < parts; ++q) {
        const uint32_t src = msrc[m + q];
        const bool fr = (src & FROM_FRAME) != 0;
        const uint32_t i = src & ~FROM_FRAME;
        const CacheArrays &s = fr ? f : c;
        const double wgt = fr ? alpha : 1.0 - alpha;
        double et = 0.0;
        for (int b = 0; b < B; ++b) {
            const double v = wgt * s.E[(size_t)i * B + b];
            E[b] += v;
            et += v;
        }
        Et += et;
        num += et * s.delay[i];
        for (int cc = 0; cc < BK; ++cc)
            out.X[(size_t)o * BK + cc] = (q == 0 ? 0.0 : out.X[(size_t)o * BK + cc]) + wgt * s.X[(size_t)i * BK + cc];
    }
    out.key[o] = mkey[m];
    for (int b = 0; b < B; ++b) out.E[(size_t)o * B + b] = E[b];
    out.delay[o] = Et > 0.0 ? num / Et : 0.0;
}

// --- 5. prioritisation -------------------------------------------------------------
// sort key: decreasing total energy (the complement of the positive double's bits);
// paths at or below the hearing threshold get the largest key and are counted apart
__global__ void k_prio_keys(CacheArrays c, int n, int B, double threshold, unsigned long long *skey,
                            uint32_t *above)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double t = 0.0;
    for (int b = 0; b < B; ++b) t += c.E[(size_t)i * B + b];
    if (t > threshold) {
        skey[i] = ~(unsigned long long)__double_as_longlong(t);
        atomicAdd(above, 1u);
    } else {
        skey[i] = ~0ull;
    }
}

__global__ void k_write_rendered(CacheArrays c, const uint32_t *order, int n_out, int B, int K,
                                 rp_er_path *out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_out) return;
    const uint32_t i = order[r];
    const unsigned long long k = c.key[i];
    rp_er_path p;
    p.source = (int32_t)(k >> (2 * ER_TRI_BITS));
    const unsigned t1 = (unsigned)((k >> ER_TRI_BITS) & ER_TRI_NONE), t2 = (unsigned)(k & ER_TRI_NONE);
    p.tri[0] = (int32_t)t1;
    p.tri[1] = t2 == ER_TRI_NONE ? -1 : (int32_t)t2;
    p.order = t2 == ER_TRI_NONE ? 1 : 2;
    p.delay_s = c.delay[i];
    for (int b = 0; b < RP_MAX_BANDS; ++b) {
        p.energy[b] = b < B ? c.E[(size_t)i * B + b] : 0.0;
        for (int kk = 0; kk < RP_MAX_SH; ++kk)
            p.sh[b][kk] = (b < B && kk < K) ? c.X[((size_t)i * B + b) * K + kk] : 0.0;
    }
    out[r] = p;
}

// the paths ranked [first, last) go into the late IR H [S][B][K][T]
__global__ void k_spill(CacheArrays c, const uint32_t *order, int first, int last, int B, int K, int T,
                        double rate, float *H)
{
    const int r = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= last) return;
    const uint32_t i = order[r];
    const double binf = floor(c.delay[i] * rate);
    if (!(binf < (double)T)) return;
    const int bin = (int)binf;
    const int s = (int)(c.key[i] >> (2 * ER_TRI_BITS));
    for (int b = 0; b < B; ++b)
        for (int kk = 0; kk < K; ++kk)
            atomicAdd(&H[(((size_t)s * B + b) * K + kk) * T + bin], (float)c.X[((size_t)i * B + b) * K + kk]);
}

__global__ void k_ir_cache(const float *__restrict__ H, float *__restrict__ C, long long n, float alpha)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        C[i] = alpha >= 1.0f ? H[i] : fmaf(alpha, H[i] - C[i], C[i]);
}

}  // namespace
}  // namespace rp

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
struct rp_er_cache {
    rp_ctx *ctx = nullptr;
    int B = 0, K = 0;
    long long n = 0;     // cached paths
    long long cap = 0;   // capacity of the path arrays
    bool first = true;   // the next update has no previous state (alpha = 1)
    CacheArrays cur = {nullptr, nullptr, nullptr, nullptr}, nxt = {nullptr, nullptr, nullptr, nullptr};
    // per-update workspace
    Buf hp, hplo, hn, hws, hrid, hprev;       // early reflections
    Buf rkey, re, rlen, rrid, ridx;           // records, their sort index
    Buf tkey, tidx, counts, offs, part;       // radix sort
    Buf head, hpos, start, frame_key, fE, fX, fdelay, mkey, msrc, keep, kpos, skey, sorder, scal;
};

namespace {

int er_ok(cudaError_t e)
{
    if (e == cudaSuccess) return RP_OK;
    return e == cudaErrorMemoryAllocation ? RP_ERR_OOM : RP_ERR_CUDA;
}

#define CKE(x)                                      \
    do {                                            \
        const cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return er_ok(e_);    \
    } while (0)

int grow(Buf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return RP_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    CKE(cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
    return RP_OK;
}

int grow_cache(rp_er_cache *c, long long need)
{
    if (need <= c->cap) return RP_OK;
    long long cap = std::max(need, c->cap * 2 + 1024);
    CacheArrays a[2];
    for (auto &x : a) {
        CKE(cudaMalloc(&x.key, sizeof(unsigned long long) * cap));
        CKE(cudaMalloc(&x.E, sizeof(double) * cap * c->B));
        CKE(cudaMalloc(&x.X, sizeof(double) * cap * c->B * c->K));
        CKE(cudaMalloc(&x.delay, sizeof(double) * cap));
    }
    cudaStream_t st = c->ctx->stream;
    if (c->n > 0) {  // the cached paths move to the new arrays
        CKE(cudaMemcpyAsync(a[0].key, c->cur.key, sizeof(unsigned long long) * c->n, cudaMemcpyDeviceToDevice, st));
        CKE(cudaMemcpyAsync(a[0].E, c->cur.E, sizeof(double) * c->n * c->B, cudaMemcpyDeviceToDevice, st));
        CKE(cudaMemcpyAsync(a[0].X, c->cur.X, sizeof(double) * c->n * c->B * c->K, cudaMemcpyDeviceToDevice, st));
        CKE(cudaMemcpyAsync(a[0].delay, c->cur.delay, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, st));
        CKE(cudaStreamSynchronize(st));
    }
    for (CacheArrays *x : {&c->cur, &c->nxt}) {
        cudaFree(x->key);
        cudaFree(x->E);
        cudaFree(x->X);
        cudaFree(x->delay);
    }
    c->cur = a[0];
    c->nxt = a[1];
    c->cap = cap;
    return RP_OK;
}

// stable sort of n 64-bit keys (low `bits` bits significant) with values; results in
// key/val (the temporaries hold the other half of each pass)
int radix_sort64(rp_er_cache *c, unsigned long long *key, uint32_t *val, int n, int bits, cudaStream_t st)
{
    if (n <= 1) return RP_OK;
    const int W = std::max(1, std::min(RS_WORKERS_MAX, (n + 255) / 256));
    const int L = (n + W - 1) / W;
    int rc;
    if ((rc = grow(c->tkey, sizeof(unsigned long long) * n)) || (rc = grow(c->tidx, sizeof(uint32_t) * n)) ||
        (rc = grow(c->counts, sizeof(uint32_t) * 256 * W)) || (rc = grow(c->offs, sizeof(uint32_t) * (256 * W + 1))) ||
        (rc = grow(c->part, sizeof(uint32_t) * scan_parts(256ull * W))))
        return rc;
    unsigned long long *k0 = key, *k1 = (unsigned long long *)c->tkey.p;
    uint32_t *v0 = val, *v1 = (uint32_t *)c->tidx.p;
    const int passes = (bits + 7) / 8;
    for (int pss = 0; pss < passes; ++pss) {
        const int shift = 8 * pss;
        k_rs64_count<<<(W + 127) / 128, 128, 0, st>>>(k0, n, shift, W, L, (uint32_t *)c->counts.p);
        launch_scan_u32((uint32_t *)c->counts.p, (uint32_t *)c->offs.p, 256 * W, (uint32_t *)c->part.p, st);
        k_rs64_scatter<<<(W + 127) / 128, 128, 0, st>>>(k0, v0, k1, v1, n, shift, W, L, (uint32_t *)c->offs.p);
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    if (k0 != key) {  // an odd number of passes: the result is in the temporaries
        CKE(cudaMemcpyAsync(key, k0, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, st));
        CKE(cudaMemcpyAsync(val, v0, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    return er_ok(cudaGetLastError());
}

template <typename T>
T read1(const void *d, cudaStream_t st)
{
    T h{};
    cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return h;
}

}  // namespace

extern "C" {

int rp_er_cache_create(rp_ctx *ctx, int32_t num_bands, int32_t sh_order, rp_er_cache **out)
{
    if (!ctx || !out || num_bands < 1 || num_bands > RP_MAX_BANDS || sh_order < 0 || sh_order > RP_MAX_SH_ORDER)
        return RP_ERR_INVALID_ARG;
    *out = nullptr;
    rp_er_cache *c = new (std::nothrow) rp_er_cache();
    if (!c) return RP_ERR_OOM;
    c->ctx = ctx;
    c->B = num_bands;
    c->K = (sh_order + 1) * (sh_order + 1);
    *out = c;
    return RP_OK;
}

int rp_er_cache_destroy(rp_er_cache *c)
{
    if (!c) return RP_ERR_INVALID_ARG;
    cudaSetDevice(c->ctx->device);
    cudaStreamSynchronize(c->ctx->stream);
    for (CacheArrays *x : {&c->cur, &c->nxt}) {
        cudaFree(x->key);
        cudaFree(x->E);
        cudaFree(x->X);
        cudaFree(x->delay);
    }
    for (Buf *b : {&c->hp, &c->hplo, &c->hn, &c->hws, &c->hrid, &c->hprev, &c->rkey, &c->re, &c->rlen, &c->rrid,
                   &c->ridx, &c->tkey, &c->tidx, &c->counts, &c->offs, &c->part, &c->head, &c->hpos, &c->start,
                   &c->frame_key, &c->fE, &c->fX, &c->fdelay, &c->mkey, &c->msrc, &c->keep, &c->kpos, &c->skey,
                   &c->sorder, &c->scal})
        if (b->p) cudaFree(b->p);
    delete c;
    return RP_OK;
}

int rp_er_cache_reset(rp_er_cache *c)
{
    if (!c) return RP_ERR_INVALID_ARG;
    c->n = 0;
    c->first = true;
    return RP_OK;
}

int rp_er_cache_read(rp_er_cache *c, rp_er_path *out, int64_t max_paths, int64_t *count)
{
    if (!c || !count || (max_paths > 0 && !out)) return RP_ERR_INVALID_ARG;
    CKE(cudaSetDevice(c->ctx->device));
    *count = c->n;
    const int n = (int)std::min<long long>(c->n, max_paths);
    if (n <= 0) return RP_OK;
    cudaStream_t st = c->ctx->stream;
    int rc;
    if ((rc = grow(c->sorder, sizeof(uint32_t) * n))) return rc;
    k_iota<<<(n + 255) / 256, 256, 0, st>>>((uint32_t *)c->sorder.p, n);
    k_write_rendered<<<(n + 127) / 128, 128, 0, st>>>(c->cur, (const uint32_t *)c->sorder.p, n, c->B, c->K, out);
    return er_ok(cudaGetLastError());
}

int rp_trace_er(rp_scene *sc, const rp_trace_params *p, const float *listener, const float *sources, int32_t S,
                float *H, rp_direct *direct, rp_trace_stats *stats, rp_er_cache *cache, const rp_er_params *ep,
                rp_er_path *rendered, int32_t *num_rendered)
{
    if (!sc || !p || !cache || !ep || !H || !rendered || !num_rendered || S < 1) return RP_ERR_INVALID_ARG;
    if (p->min_order < 2 || p->min_order > 3 || p->budget_refill < 0 || cache->ctx != sc->ctx ||
        cache->B != sc->B || cache->K != (p->sh_order + 1) * (p->sh_order + 1) || ep->n_er < 0 ||
        !(ep->dt_update >= 0.0) || !(ep->tau_er >= 0.0) || !(ep->prune >= 0.0) || !(ep->hearing_threshold >= 0.0) ||
        sc->num_tris >= (int)ER_TRI_NONE || S >= (1 << 12) || (p->flags & RP_FLAG_RAY_HASH))
        return RP_ERR_INVALID_ARG;
    rp_ctx *c = sc->ctx;
    CKE(cudaSetDevice(c->device));
    cudaStream_t st = c->stream;
    const int B = sc->B, K = cache->K, T = p->num_bins;
    // early reflections: at most min_order - 1 per primary, and never more than the
    // step's N x M segments (the bound with budget refill)
    const unsigned long long ecap = std::max(
        1ull, p->num_rays * (unsigned long long)std::max(1, p->budget_refill ? p->max_order
                                                                              : std::min(p->max_order, p->min_order - 1)));
    int rc;
    if ((rc = grow(cache->hp, sizeof(float4) * ecap)) || (rc = grow(cache->hplo, sizeof(float4) * ecap)) ||
        (rc = grow(cache->hn, sizeof(float4) * ecap)) || (rc = grow(cache->hws, sizeof(float) * ecap * B)) ||
        (rc = grow(cache->hrid, sizeof(uint32_t) * ecap)) || (rc = grow(cache->hprev, sizeof(int) * ecap)))
        return rc;
    EarlyHits eh;
    eh.hits = {(float4 *)cache->hp.p, (float4 *)cache->hplo.p, (float4 *)cache->hn.p, (float *)cache->hws.p,
               (uint32_t *)cache->hrid.p, ecap};
    eh.prev = (int *)cache->hprev.p;
    eh.cap = ecap;
    TraceWork w;
    if ((rc = trace_enqueue(sc, p, listener, sources, S, H, direct, stats, nullptr, &eh, &w))) return rc;

    // 2. early-reflection shadow rays -> records
    const unsigned long long n_er = std::min(read1<unsigned long long>(&w.ctr->n_er, st), ecap);
    const unsigned long long rcap = std::max(1ull, n_er * (unsigned long long)S);
    if (rcap > 0x7fffffffull) return RP_ERR_TOO_LARGE;
    if ((rc = grow(cache->rkey, sizeof(unsigned long long) * rcap)) || (rc = grow(cache->re, sizeof(float) * rcap * B)) ||
        (rc = grow(cache->rlen, sizeof(double) * rcap)) || (rc = grow(cache->rrid, sizeof(uint32_t) * rcap)) ||
        (rc = grow(cache->ridx, sizeof(uint32_t) * rcap)) || (rc = grow(cache->scal, 64)))
        return rc;
    unsigned long long *rcount = (unsigned long long *)cache->scal.p;
    CKE(cudaMemsetAsync(rcount, 0, 64, st));
    if (n_er > 0)
        k_er_shadow<<<c->num_sms * 8, ER_THREADS, 0, st>>>(w, (unsigned long long *)cache->rkey.p, (float *)cache->re.p,
                                                           (double *)cache->rlen.p, (uint32_t *)cache->rrid.p, rcap,
                                                           rcount);
    CKE(cudaGetLastError());
    const int nrec = (int)std::min<unsigned long long>(read1<unsigned long long>(rcount, st), rcap);

    // 3. sort by key, one path per key
    unsigned long long *rkey = (unsigned long long *)cache->rkey.p;
    uint32_t *ridx = (uint32_t *)cache->ridx.p;
    int P = 0;
    if (nrec > 0) {
        k_iota<<<(nrec + 255) / 256, 256, 0, st>>>(ridx, nrec);
        if ((rc = radix_sort64(cache, rkey, ridx, nrec, (int)(2 * ER_TRI_BITS + 12), st))) return rc;
        if ((rc = grow(cache->head, sizeof(uint32_t) * nrec)) || (rc = grow(cache->hpos, sizeof(uint32_t) * (nrec + 1))) ||
            (rc = grow(cache->start, sizeof(uint32_t) * (nrec + 1))) ||
            (rc = grow(cache->part, sizeof(uint32_t) * scan_parts((unsigned long long)std::max(nrec, 256 * RS_WORKERS_MAX)))))
            return rc;
        k_heads<<<(nrec + 255) / 256, 256, 0, st>>>(rkey, nrec, (uint32_t *)cache->head.p);
        launch_scan_u32((uint32_t *)cache->head.p, (uint32_t *)cache->hpos.p, nrec, (uint32_t *)cache->part.p, st);
        k_starts<<<(nrec + 255) / 256, 256, 0, st>>>((uint32_t *)cache->head.p, (uint32_t *)cache->hpos.p, nrec,
                                                    (uint32_t *)cache->start.p);
        P = (int)read1<uint32_t>((uint32_t *)cache->hpos.p + nrec, st);
    }
    if ((rc = grow(cache->frame_key, sizeof(unsigned long long) * std::max(P, 1))) ||
        (rc = grow(cache->fE, sizeof(double) * std::max(P, 1) * B)) ||
        (rc = grow(cache->fX, sizeof(double) * std::max(P, 1) * B * K)) ||
        (rc = grow(cache->fdelay, sizeof(double) * std::max(P, 1))))
        return rc;
    CacheArrays fr = {(unsigned long long *)cache->frame_key.p, (double *)cache->fE.p, (double *)cache->fX.p,
                      (double *)cache->fdelay.p};
    if (P > 0)
        k_path_reduce<<<std::min((P + 3) / 4, c->num_sms * 16), 128, 0, st>>>(
            w, rkey, ridx, (uint32_t *)cache->start.p, (uint32_t *)cache->hpos.p + nrec, (float *)cache->re.p,
            (double *)cache->rlen.p, (uint32_t *)cache->rrid.p, fr.key, fr.E, fr.X, fr.delay);
    CKE(cudaGetLastError());

    // 4. merge with the cache
    const double alpha = (cache->first || !(ep->tau_er > 0.0)) ? 1.0 : 1.0 - std::exp(-ep->dt_update / ep->tau_er);
    const long long nc = cache->n, nm = nc + P;
    if ((rc = grow_cache(cache, nm))) return rc;
    if ((rc = grow(cache->mkey, sizeof(unsigned long long) * std::max(nm, 1ll))) ||
        (rc = grow(cache->msrc, sizeof(uint32_t) * std::max(nm, 1ll))) ||
        (rc = grow(cache->keep, sizeof(uint32_t) * std::max(nm, 1ll))) ||
        (rc = grow(cache->kpos, sizeof(uint32_t) * (nm + 1))) ||
        (rc = grow(cache->part, sizeof(uint32_t) * scan_parts((unsigned long long)std::max<long long>(nm, 256 * RS_WORKERS_MAX)))))
        return rc;
    long long nn = 0;
    if (nm > 0) {
        const int g = (int)((nm + 255) / 256);
        k_merge_pos<<<g, 256, 0, st>>>(cache->cur.key, (int)nc, fr.key, P, (unsigned long long *)cache->mkey.p,
                                       (uint32_t *)cache->msrc.p);
        k_merge_flags<<<g, 256, 0, st>>>((unsigned long long *)cache->mkey.p, (uint32_t *)cache->msrc.p, (int)nm,
                                         cache->cur, fr, B, alpha, ep->prune, (uint32_t *)cache->keep.p);
        launch_scan_u32((uint32_t *)cache->keep.p, (uint32_t *)cache->kpos.p, (int)nm, (uint32_t *)cache->part.p, st);
        k_merge_write<<<g, 256, 0, st>>>((unsigned long long *)cache->mkey.p, (uint32_t *)cache->msrc.p, (int)nm,
                                         (uint32_t *)cache->keep.p, (uint32_t *)cache->kpos.p, cache->cur, fr, B, B * K,
                                         alpha, cache->nxt);
        nn = (long long)read1<uint32_t>((uint32_t *)cache->kpos.p + nm, st);
    }
    std::swap(cache->cur, cache->nxt);
    cache->n = nn;
    cache->first = false;

    // 5. prioritisation: rendered paths, and the rest into the late IR
    int n_out = 0;
    if (nn > 0) {
        if ((rc = grow(cache->skey, sizeof(unsigned long long) * nn)) || (rc = grow(cache->sorder, sizeof(uint32_t) * nn)))
            return rc;
        uint32_t *above = (uint32_t *)cache->scal.p + 4;
        CKE(cudaMemsetAsync(above, 0, sizeof(uint32_t), st));
        k_prio_keys<<<(int)((nn + 255) / 256), 256, 0, st>>>(cache->cur, (int)nn, B, ep->hearing_threshold,
                                                             (unsigned long long *)cache->skey.p, above);
        k_iota<<<(int)((nn + 255) / 256), 256, 0, st>>>((uint32_t *)cache->sorder.p, (int)nn);
        if ((rc = radix_sort64(cache, (unsigned long long *)cache->skey.p, (uint32_t *)cache->sorder.p, (int)nn, 64, st)))
            return rc;
        const int A = (int)read1<uint32_t>(above, st);
        n_out = std::min(A, ep->n_er);
        if (n_out > 0)
            k_write_rendered<<<(n_out + 127) / 128, 128, 0, st>>>(cache->cur, (uint32_t *)cache->sorder.p, n_out, B, K,
                                                                  rendered);
        if (A > n_out)
            k_spill<<<(A - n_out + 127) / 128, 128, 0, st>>>(cache->cur, (uint32_t *)cache->sorder.p, n_out, A, B, K,
                                                             T, (double)p->ir_rate_hz, H);
    }
    CKE(cudaMemcpyAsync(num_rendered, &n_out, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CKE(cudaStreamSynchronize(st));  // n_out lives on this stack frame
    return er_ok(cudaGetLastError());
}

int rp_ir_cache_update(rp_ctx *c, const float *H, float *C, int64_t count, double dt_update, double tau, int32_t first)
{
    if (!c || !H || !C || count < 0 || !(dt_update >= 0.0) || !(tau >= 0.0)) return RP_ERR_INVALID_ARG;
    CKE(cudaSetDevice(c->device));
    const double alpha = (first || !(tau > 0.0)) ? 1.0 : 1.0 - std::exp(-dt_update / tau);
    if (count == 0) return RP_OK;
    const long long nb = std::min<long long>((count + 255) / 256, (long long)c->num_sms * 16);
    k_ir_cache<<<(int)nb, 256, 0, c->stream>>>(H, C, count, (float)alpha);
    return er_ok(cudaGetLastError());
}

}  // extern "C"
