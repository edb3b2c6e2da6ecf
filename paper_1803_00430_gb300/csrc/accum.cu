// accum.cu -- binning of contribution records into the low-rate SH energy
// histogram H[s][b][k][t] (Section 4.2: I_b(t) with its spherical-harmonic
// directivity X_{b,lm}(t); arrival direction = the path's first segment).
//
// Records (key = source * T + bin, primary ray id, e[B]) are grouped by key with a
// counting sort (count, exclusive scan, scatter of record indices).  Then one warp
// owns one (source, bin): its 32 lanes own the B*K cells, 32 records at a time are
// staged in shared memory (energies, and SH of the primary direction recomputed
// from Philox), and every cell is summed in FP32: each group of 32 staged records
// with plain fused multiply-adds (relative error at most 32 * 2^-24), the groups with
// Kahan compensation.  A key with more than ACC_SEG records in a chunk is split into
// segments of ACC_SEG records, each summed so by its own warp, and its warp then
// combines the segments' pairs in segment order with an error-free two-sum: a few
// keys can hold a large share of the records (one warp each left most of the GPU idle
// while they finished), and the fixed segmentation keeps the sums deterministic.
// Each cell is written by exactly one warp, so no atomics touch H.  Chunks of records (when the record buffer is smaller than one step's records)
// are merged into a running (sum, error) pair with an error-free two-sum.  The running
// pair is kept key-major, [source][bin][band][coefficient], so that a warp's B*K cells
// of one key are contiguous (coalesced loads and stores); the finalize kernel
// transposes it through shared memory into H[s][b][k][t].
#include "internal.cuh"

namespace rp {
namespace {

constexpr int ACC_THREADS = 256;
constexpr int ACC_WARPS = ACC_THREADS / 32;
constexpr int ACC_SLOTS = (MAXB * MAXK + 31) / 32;

// Record chunks are sized for the worst case (every primary reflecting M times);
// a chunk past the step's actual shadow items has no records and is skipped on the
// device.  Chunk 0 always runs: it also holds the source-sphere records of the paths.
__device__ __forceinline__ bool chunk_active(const TraceWork &w, unsigned long long chunk)
{
    return chunk == 0 || chunk * w.items_per_chunk < w.ctr->total_items;
}

__global__ void k_clear_counts(TraceWork w, unsigned long long chunk)
{
    if (!chunk_active(w, chunk)) return;
    const long long n = (long long)w.k.S * w.k.T;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        w.cnt[i] = 0u;
        w.cur[i] = 0u;
    }
}

// a source-sphere record of a ray past the waves of a store pass (chunk 0 holds them)
__device__ __forceinline__ bool dropped_record(const TraceWork &w, unsigned long long i)
{
    return (unsigned long long)w.rec.rid[i] >= w.rid_end;
}

__global__ void k_count(TraceWork w, unsigned long long chunk)
{
    if (!chunk_active(w, chunk)) return;
    const unsigned long long n = min(w.ctr->n_records, w.rec.cap);
    const bool drop = w.rid_end && chunk == 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        if (drop && dropped_record(w, i)) continue;
        if (RP_IN_RANGE(w.rec.key[i], (unsigned long long)w.k.S * w.k.T, w.status)) atomicAdd(&w.cnt[w.rec.key[i]], 1u);
    }
}

// Exclusive scan of cnt[0..n) into off[0..n] (off[n] = total; off may be cnt).  A
// block of 1024 threads scans tiles of SCAN_TILE = 4096 counts, each thread taking 4
// consecutive ones.  Short arrays take one block that walks the tiles carrying the
// running total; long ones take two launches: the tile sums, then every tile scanned
// in parallel from its carry, which its block adds up from the sums of the tiles
// before it.  With a gate, the scan is skipped when *gate_total <= gate_q0 (an empty
// record chunk).
__device__ __forceinline__ bool scan_gated(const unsigned long long *gate_total, unsigned long long gate_q0)
{
    return gate_total && gate_q0 > 0 && *gate_total <= gate_q0;
}

// scan of the tile at `base` from `carry`; returns the tile's total (every thread)
__device__ __forceinline__ uint32_t scan_tile(const uint32_t *cnt, uint32_t *off, int n, int base, uint32_t carry,
                                              uint32_t *warp_sums)
{
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int i0 = base + 4 * t;
    uint32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = i0 + k < n ? cnt[i0 + k] : 0u;
        s += v[k];
    }
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t ws = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, ws, o);
            if (lane >= o) ws += y;
        }
        warp_sums[lane] = ws;
    }
    __syncthreads();
    uint32_t run = carry + x - s + (wid > 0 ? warp_sums[wid - 1] : 0u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (i0 + k < n) off[i0 + k] = run;
        run += v[k];
    }
    const uint32_t total = warp_sums[31];
    __syncthreads();  // every thread has read warp_sums
    return total;
}

__global__ void __launch_bounds__(1024) k_scan(const uint32_t *cnt, uint32_t *off, int n,
                                               const unsigned long long *gate_total, unsigned long long gate_q0)
{
    if (scan_gated(gate_total, gate_q0)) return;
    __shared__ uint32_t warp_sums[32];
    uint32_t carry = 0;
    for (int base = 0; base < n; base += SCAN_TILE) carry += scan_tile(cnt, off, n, base, carry, warp_sums);
    if (threadIdx.x == 0) off[n] = carry;
}

// sum of part[0..m) over the block (every thread gets it)
__device__ __forceinline__ uint32_t block_sum(const uint32_t *part, int m, uint32_t *warp_sums)
{
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    uint32_t s = 0;
    for (int i = t; i < m; i += blockDim.x) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) warp_sums[wid] = s;
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_sums[w];
    __syncthreads();  // warp_sums is reused
    return tot;
}

// sum of each tile
__global__ void __launch_bounds__(1024) k_scan_part(const uint32_t *cnt, int n, uint32_t *part,
                                                    const unsigned long long *gate_total, unsigned long long gate_q0)
{
    if (scan_gated(gate_total, gate_q0)) return;
    __shared__ uint32_t warp_sums[32];
    const int i0 = blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = i0 + k < n ? cnt[i0 + k] : 0u;
    // the four counts of each thread, then the block
    __shared__ uint32_t sums[1024];
    sums[threadIdx.x] = v[0] + v[1] + v[2] + v[3];
    __syncthreads();
    const uint32_t tot = block_sum(sums, 1024, warp_sums);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// every tile from its carry, the sum of the tiles before it (part: the tile sums)
__global__ void __launch_bounds__(1024) k_scan_apply(const uint32_t *cnt, uint32_t *off, int n,
                                                     const uint32_t *part, int nparts,
                                                     const unsigned long long *gate_total, unsigned long long gate_q0)
{
    if (scan_gated(gate_total, gate_q0)) return;
    __shared__ uint32_t warp_sums[32];
    const uint32_t carry = block_sum(part, blockIdx.x, warp_sums);
    if (blockIdx.x == 0) {
        const uint32_t total = block_sum(part, nparts, warp_sums);
        if (threadIdx.x == 0) off[n] = total;
    }
    scan_tile(cnt, off, n, blockIdx.x * SCAN_TILE, carry, warp_sums);
}

__global__ void k_scatter(TraceWork w, unsigned long long chunk)
{
    if (!chunk_active(w, chunk)) return;
    const unsigned long long n = min(w.ctr->n_records, w.rec.cap);
    const bool drop = w.rid_end && chunk == 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        if (drop && dropped_record(w, i)) continue;
        const uint32_t key = w.rec.key[i];
        if (!RP_IN_RANGE(key, (unsigned long long)w.k.S * w.k.T, w.status)) continue;
        const uint32_t pos = w.off[key] + atomicAdd(&w.cur[key], 1u);
        if (RP_IN_RANGE(pos, w.rec.cap, w.status)) w.perm[pos] = (uint32_t)i;
    }
}

// Kahan step with the error kept as "true minus sum"
__device__ __forceinline__ void kahan_add(float &sum, float &err, float x)
{
    const float y = __fadd_rn(x, err);
    const float t = __fadd_rn(sum, y);
    err = __fsub_rn(y, __fsub_rn(t, sum));
    sum = t;
}

// The compensated sums of records perm[begin .. end) of one key, by one warp: lane l
// owns cells l + 32 i; groups of 32 records are staged in shared memory (energies and
// the SH of the primary direction), summed in plain FP32, and the groups Kahan-added.
__device__ __forceinline__ void accum_range(const TraceWork &w, long long key, uint32_t begin, uint32_t end,
                                            float (*se)[MAXB], float (*sy)[MAXK], float *sum, float *err)
{
    const int lane = threadIdx.x & 31;
    const int B = w.k.B, K = w.k.K, T = w.k.T, BK = B * K;
    const unsigned long long seed = w.seed ? w.seed[0] : w.seed_val;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const int gs = w.src_base + (int)(key / T);
    const uint32_t scene_id = w.njobs > 1 ? w.jobs[w.src_job[gs]].scene_id : w.job0.scene_id;
#pragma unroll
    for (int i = 0; i < ACC_SLOTS; ++i) sum[i] = err[i] = 0.f;
    for (uint32_t base = begin; base < end; base += 32) {
        const int n = (int)min(32u, end - base);
        if (lane < n) {
            uint32_t r = w.perm[base + lane];
            if (!RP_IN_RANGE(r, w.rec.cap, w.status)) r = 0;  // (checked build) keep going on record 0
            const uint32_t rid = w.rec.rid[r];
            const float *e = w.rec.e + (unsigned long long)r * B;
#pragma unroll
            for (int b = 0; b < MAXB; ++b)
                if (b < B) se[lane][b] = e[b];
            const float3 d0 = primary_direction(rid, scene_id, key0, key1);
            float Y[MAXK];
            sh_eval(w.k.sh_order, d0.x, d0.y, d0.z, Y);
#pragma unroll
            for (int kk = 0; kk < MAXK; ++kk)
                if (kk < K) sy[lane][kk] = Y[kk];
        }
        __syncwarp();
        // the staged records in plain FP32, then one compensated add per group of 32
        float part[ACC_SLOTS];
#pragma unroll
        for (int i = 0; i < ACC_SLOTS; ++i) part[i] = 0.f;
#pragma unroll
        for (int i = 0; i < ACC_SLOTS; ++i) {
            const int c = lane + 32 * i;
            if (c < BK) {
                const int b = c / K, kk = c - b * K;
                for (int j = 0; j < n; ++j) part[i] = fmaf(se[j][b], sy[j][kk], part[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < ACC_SLOTS; ++i) kahan_add(sum[i], err[i], part[i]);
        __syncwarp();
    }
}

// two-sum merge of the pair (b, be) into the running pair (a, ae)
__device__ __forceinline__ void pair_merge(float &a, float &ae, float b, float be)
{
    const float s2 = __fadd_rn(a, b);
    const float bp = __fsub_rn(s2, a);
    const float e2 = __fadd_rn(__fsub_rn(a, __fsub_rn(s2, bp)), __fsub_rn(b, bp));
    a = s2;
    ae = ae + be + e2;
}

// Heavy keys: cur[key] = its number of segments of ACC_SEG records when it has more
// than ACC_SEG records in this chunk, else 0 (its warp in k_accum sums it directly).
__global__ void k_seg_count(TraceWork w, unsigned long long chunk)
{
    if (!chunk_active(w, chunk)) return;
    const long long n = (long long)w.k.S * w.k.T;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = w.off[i + 1] - w.off[i];
        w.cur[i] = c > ACC_SEG ? (c + ACC_SEG - 1) / ACC_SEG : 0u;
    }
}

// after the scan of cur into cnt: the key of every segment
__global__ void k_seg_map(TraceWork w, unsigned long long chunk)
{
    if (!chunk_active(w, chunk)) return;
    const long long n = (long long)w.k.S * w.k.T;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t m = w.cur[i], g0 = w.cnt[i];
        for (uint32_t j = 0; j < m; ++j) {
            if ((unsigned long long)g0 + j >= w.seg_cap) {  // cannot happen: seg_cap holds 2 rec_cap / ACC_SEG
                raise_error(w.status, RP_ERR_CAPACITY);
                break;
            }
            w.segkey[g0 + j] = (uint32_t)i;
        }
    }
}

// one warp per segment of a heavy key: its compensated sums into Ss / Se
__global__ void __launch_bounds__(ACC_THREADS) k_accum_seg(TraceWork w, unsigned long long chunk)
{
    if (!chunk_active(w, chunk)) return;
    __shared__ float se[ACC_WARPS][32][MAXB];
    __shared__ float sy[ACC_WARPS][32][MAXK];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long nkeys = (long long)w.k.S * w.k.T;
    const int BK = w.k.B * w.k.K;
    const unsigned long long nseg = min((unsigned long long)w.cnt[nkeys], w.seg_cap);
    const unsigned long long nwarps = (unsigned long long)gridDim.x * ACC_WARPS;
    for (unsigned long long g = (unsigned long long)blockIdx.x * ACC_WARPS + wp; g < nseg; g += nwarps) {
        const uint32_t key = w.segkey[g];
        if (key >= (unsigned long long)nkeys) continue;
        const uint32_t begin = w.off[key] + (uint32_t)(g - w.cnt[key]) * ACC_SEG;
        const uint32_t end = min(begin + ACC_SEG, w.off[key + 1]);
        float sum[ACC_SLOTS], err[ACC_SLOTS];
        accum_range(w, key, begin, end, se[wp], sy[wp], sum, err);
#pragma unroll
        for (int i = 0; i < ACC_SLOTS; ++i) {
            const int c = lane + 32 * i;
            if (c < BK) {
                w.Ss[g * BK + c] = sum[i];
                w.Se[g * BK + c] = err[i];
            }
        }
    }
}

// One warp per (source, bin): this chunk's sums of the key -- its records directly,
// or its segments' sums (k_accum_seg) combined in segment order -- merged into the
// running pair (written on the first chunk).
__global__ void __launch_bounds__(ACC_THREADS) k_accum(TraceWork w, int first, unsigned long long chunk)
{
    if (!chunk_active(w, chunk)) return;
    __shared__ float se[ACC_WARPS][32][MAXB];
    __shared__ float sy[ACC_WARPS][32][MAXK];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int S = w.k.S, B = w.k.B, K = w.k.K, T = w.k.T, BK = B * K;
    const long long nkeys = (long long)S * T;
    const long long nwarps = (long long)gridDim.x * ACC_WARPS;
    for (long long key = (long long)blockIdx.x * ACC_WARPS + wp; key < nkeys; key += nwarps) {
        const uint32_t begin = w.off[key], end = w.off[key + 1];
        if (!first && begin == end) continue;  // nothing to merge: the running pair stands
        float sum[ACC_SLOTS], err[ACC_SLOTS];
        const uint32_t m = w.cur[key];
        if (m == 0) {
            accum_range(w, key, begin, end, se[wp], sy[wp], sum, err);
        } else {
            const unsigned long long g0 = w.cnt[key];
#pragma unroll
            for (int i = 0; i < ACC_SLOTS; ++i) sum[i] = err[i] = 0.f;
            for (uint32_t j = 0; j < m; ++j) {
                const unsigned long long g = g0 + j;
                if (g >= w.seg_cap) break;  // (k_seg_map has raised the error)
#pragma unroll
                for (int i = 0; i < ACC_SLOTS; ++i) {
                    const int c = lane + 32 * i;
                    if (c < BK) {
                        if (j == 0) {
                            sum[i] = w.Ss[g * BK + c];
                            err[i] = w.Se[g * BK + c];
                        } else {
                            pair_merge(sum[i], err[i], w.Ss[g * BK + c], w.Se[g * BK + c]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < ACC_SLOTS; ++i) {
            const int c = lane + 32 * i;
            if (c < BK) {
                // running pair, key-major: [s][bin][b][kk]
                const unsigned long long idx = (unsigned long long)key * BK + c;
                if (!RP_IN_RANGE(idx, (unsigned long long)S * B * K * T, w.status)) continue;
                if (first) {
                    w.Hs[idx] = sum[i];
                    w.He[idx] = err[i];
                } else {
                    float a = w.Hs[idx], ae = w.He[idx];
                    pair_merge(a, ae, sum[i], err[i]);
                    w.Hs[idx] = a;
                    w.He[idx] = ae;
                }
            }
        }
    }
}

// H[s][b][k][t] = (sum + error)[s][t][b][k] / K_primaries of the source's job: a 32 x 32
// tile of (bin, cell) per block, read along cells and written along bins through shared
// memory.  Block (0, 0, 0) also normalises the late energy (one job).
constexpr int FIN_TILE = 32;

__global__ void __launch_bounds__(FIN_TILE * 8) k_finalize(TraceWork w)
{
    __shared__ float tile[FIN_TILE][FIN_TILE + 1];
    const int BK = w.k.B * w.k.K, T = w.k.T;
    const int t0 = blockIdx.x * FIN_TILE, c0 = blockIdx.y * FIN_TILE;
    const int tx = threadIdx.x & (FIN_TILE - 1), ty = threadIdx.x / FIN_TILE;
    const unsigned long long src_cells = (unsigned long long)BK * T;
    for (int s = blockIdx.z; s < w.k.S; s += gridDim.z) {
        const int gs = w.src_base + s;
        const unsigned long long kp = w.njobs > 1 ? w.js[w.src_job[gs]].primaries : w.js[0].primaries;
        const float *hs = w.Hs + (unsigned long long)s * src_cells;
        const float *he = w.He + (unsigned long long)s * src_cells;
        __syncthreads();  // the previous source's tile has been written out
        for (int r = ty; r < FIN_TILE; r += 8) {  // r: bin within the tile, tx: cell
            const int t = t0 + r, c = c0 + tx;
            float v = 0.f;
            if (t < T && c < BK && kp > 0) {
                const unsigned long long i = (unsigned long long)t * BK + c;
                v = (hs[i] + he[i]) / (float)kp;
            }
            tile[r][tx] = v;
        }
        __syncthreads();
        float *Hg = w.H + ((unsigned long long)gs * BK) * T;
        for (int r = ty; r < FIN_TILE; r += 8) {  // r: cell within the tile, tx: bin
            const int c = c0 + r, t = t0 + tx;
            if (t < T && c < BK) Hg[(unsigned long long)c * T + t] = tile[tx][r];
        }
    }
    if (w.njobs == 1 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x < w.k.B &&
        w.js[0].primaries > 0)
        w.stats->late[threadIdx.x] /= (double)w.js[0].primaries;
}

__global__ void k_direct_add(TraceWork w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int S = w.k.S, B = w.k.B, K = w.k.K, T = w.k.T;
    if (i >= S * B * K) return;
    const int s = i / (B * K), r = i - s * B * K, kk = r - (r / K) * K;
    const int gs = w.src_base + s;
    const rp_direct dd = w.direct[gs];
    if (!dd.visible || dd.bin < 0 || dd.bin >= T) return;
    w.H[((unsigned long long)w.src_base * B * K + i) * T + dd.bin] += dd.sh[kk];
}

void scan_u32(const uint32_t *cnt, uint32_t *off, int n, uint32_t *part, const unsigned long long *gate_total,
              unsigned long long gate_q0, cudaStream_t st)
{
    const int nparts = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (!part || nparts <= 2) {
        k_scan<<<1, 1024, 0, st>>>(cnt, off, n, gate_total, gate_q0);
        return;
    }
    k_scan_part<<<nparts, 1024, 0, st>>>(cnt, n, part, gate_total, gate_q0);
    k_scan_apply<<<nparts, 1024, 0, st>>>(cnt, off, n, part, nparts, gate_total, gate_q0);
}

}  // namespace

void launch_clear_counts(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st)
{
    k_clear_counts<<<blocks, 256, 0, st>>>(w, chunk);
}

void launch_count(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st)
{
    k_count<<<blocks, 256, 0, st>>>(w, chunk);
}

void launch_scan_u32(const uint32_t *cnt, uint32_t *off, int n, uint32_t *part, cudaStream_t st)
{
    scan_u32(cnt, off, n, part, nullptr, 0ull, st);
}

void launch_scan(const TraceWork &w, unsigned long long chunk, cudaStream_t st)
{
    scan_u32(w.cnt, w.off, w.k.S * w.k.T, w.scan_part, &w.ctr->total_items, chunk * w.items_per_chunk, st);
}

void launch_scatter(const TraceWork &w, unsigned long long chunk, int blocks, cudaStream_t st)
{
    k_scatter<<<blocks, 256, 0, st>>>(w, chunk);
}

void launch_accum(const TraceWork &w, int first_chunk, unsigned long long chunk, int blocks, cudaStream_t st)
{
    // heavy keys: their segments, the segments' keys, then a warp per segment
    const int n = w.k.S * w.k.T;
    const int kb = std::min((n + 255) / 256, 4 * std::max(w.num_sms, 1) * 8);
    k_seg_count<<<kb, 256, 0, st>>>(w, chunk);
    scan_u32(w.cur, w.cnt, n, w.scan_part, &w.ctr->total_items, chunk * w.items_per_chunk, st);
    k_seg_map<<<kb, 256, 0, st>>>(w, chunk);
    k_accum_seg<<<blocks, ACC_THREADS, 0, st>>>(w, chunk);
    k_accum<<<blocks, ACC_THREADS, 0, st>>>(w, first_chunk, chunk);
}

void launch_finalize(const TraceWork &w, cudaStream_t st)
{
    const int BK = w.k.B * w.k.K;
    const dim3 grid((w.k.T + FIN_TILE - 1) / FIN_TILE, (BK + FIN_TILE - 1) / FIN_TILE, std::min(w.k.S, 65535));
    if (w.k.S > 0) k_finalize<<<grid, FIN_TILE * 8, 0, st>>>(w);
    if (w.k.min_order == 0 && w.direct) {
        const int m = w.k.S * w.k.B * w.k.K;
        k_direct_add<<<(m + 255) / 256, 256, 0, st>>>(w);
    }
}

}  // namespace rp
