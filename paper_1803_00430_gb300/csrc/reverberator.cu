// reverberator.cu -- the SH-domain Schroeder reverberator of Section 4.1 ("Sound
// Rendering"), rendered on the GPU for many sources at once, block by block with its
// state kept in device memory between blocks:
//   k_rv_bands    a warp per source: the serial Linkwitz-Riley 4th-order crossover
//                 (2nd-order Butterworth biquads applied twice, transposed direct form
//                 II in FP64), the block cut into 32 chunks that run in parallel from
//                 chunk-start states found by a scan (k_rv_phi: the L-sample transition);
//   k_rv_predelay the band signals read at the predelay (this block or the ring);
//   k_rv_combs    a block per (source, band): the N_comb comb filters of the band, each
//                 a ring of K-vectors, y[n] = comb_in x[n] + g J y[n - d] (the feedback
//                 sample rotated by the comb's SH rotation and scaled by its gain), in
//                 chunks of d parallel samples, summed;
//   k_rv_allpass  a warp per (source, band, SH channel): the 4 all-pass filters in
//                 series, v[n] = -a u[n] + u[n - d] + a v[n - d], in shared memory;
//   k_rv_out      a thread per (source, sample): q = sum_b g_reverb_b D_b v_b (the
//                 directional loudness matrix and the reverberator gain of each band);
//   k_rv_advance  the sample counter of every source.
// Rings are indexed by the absolute sample number modulo their length, so the comb
// delays may change between blocks (when they are drawn again) without moving data.
#include <cmath>

#include "handles.cuh"

using namespace rp;

namespace rp {
namespace {

constexpr int N_AP = 4;
constexpr double AP_GAIN = 0.7;
constexpr double AP_MS[N_AP] = {5.0, 1.7, 0.6, 0.2};
constexpr int MAXX = RP_MAX_BANDS - 1;  // crossovers
constexpr int AP_SEG = 1024;             // all-pass segment (samples in shared memory)
constexpr int AP_WARPS = 4;              // all-pass warps per block

struct Biquad {
    double b0, b1, b2, a1, a2;
};

struct RvShape {
    int S, B, K, N, Dmax, Pmax;
    int ap_d[N_AP], ap_off[N_AP], ap_len, ap_h;  // all-pass delays (samples), ring offsets, longest delay
    double fs;
    Biquad lp[MAXX], hp[MAXX];
    // per-source state layout (bytes from the source's base)
    size_t off_x, off_n0, off_pre, off_comb, off_ap, bytes;
};

// 2nd-order Butterworth biquad by the bilinear transform (crossover frequency prewarped)
Biquad butterworth2(double fc, double fs, bool high)
{
    const double k = std::tan(3.141592653589793 * fc / fs), q = std::sqrt(2.0);
    const double norm = 1.0 / (1.0 + q * k + k * k);
    Biquad f;
    f.a1 = 2.0 * (k * k - 1.0) * norm;
    f.a2 = (1.0 - q * k + k * k) * norm;
    if (high) {
        f.b0 = norm;
        f.b1 = -2.0 * norm;
        f.b2 = norm;
    } else {
        f.b0 = k * k * norm;
        f.b1 = 2.0 * f.b0;
        f.b2 = f.b0;
    }
    return f;
}

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

void layout(RvShape &sh)
{
    size_t o = 0;
    sh.off_x = o;  // crossover states: [crossover][lp, hp][section][z1, z2] doubles
    o = align16(o + sizeof(double) * (size_t)std::max(sh.B - 1, 0) * 2 * 2 * 2);
    sh.off_n0 = o;
    o = align16(o + sizeof(long long));
    sh.off_pre = o;  // [Pmax + 1][B] floats
    o = align16(o + sizeof(float) * (size_t)(sh.Pmax + 1) * sh.B);
    sh.off_comb = o;  // [B][N_COMB][Dmax][K] floats
    o = align16(o + sizeof(float) * (size_t)sh.B * RP_N_COMB * sh.Dmax * sh.K);
    sh.off_ap = o;  // [B][K][ap_len] floats
    o = align16(o + sizeof(float) * (size_t)sh.B * sh.K * sh.ap_len);
    sh.bytes = o;
}

__device__ __forceinline__ double biquad_step(const Biquad &f, double *z, double x)
{
    const double y = f.b0 * x + z[0];
    z[0] = f.b1 * x - f.a1 * y + z[1];
    z[1] = f.b2 * x - f.a2 * y;
    return y;
}

__device__ __forceinline__ int delay_samples(double t, double fs)
{
    return isfinite(t) ? (int)fmax(0.0, floor(t * fs + 0.5)) : 0;
}

// the crossover tree at one sample: band b < B-1 is the LR4 low-pass of what the earlier
// high-passes left, the last band the final high-pass; z holds [lp1 lp2 hp1 hp2] x
// (z1, z2) for each crossover
template <int NB>
__device__ __forceinline__ void tree_step(const RvShape &sh, double *z, double x, double *y)
{
    double rest = x;
#pragma unroll
    for (int b = 0; b < NB - 1; ++b) {
        double *zb = z + b * 8;
        y[b] = biquad_step(sh.lp[b], zb + 2, biquad_step(sh.lp[b], zb, rest));
        rest = biquad_step(sh.hp[b], zb + 6, biquad_step(sh.hp[b], zb + 4, rest));
    }
    y[NB - 1] = rest;
}

// Phi = A^L, the tree's state after L samples of zero input from each unit state
// (column c from state e_c), for the chunk scan of k_rv_bands
template <int NB>
__global__ void k_rv_phi(RvShape sh, int L, double *__restrict__ phi)
{
    constexpr int M = 8 * (NB - 1);
    const int c = threadIdx.x;
    if (M == 0 || c >= M) return;
    double z[M > 0 ? M : 1], y[NB];
#pragma unroll
    for (int r = 0; r < M; ++r) z[r] = r == c ? 1.0 : 0.0;
    for (int n = 0; n < L; ++n) tree_step<NB>(sh, z, 0.0, y);
#pragma unroll
    for (int r = 0; r < M; ++r) phi[r * M + c] = z[r];
}

// the crossover, a warp per source, in FP64: the block is cut into 32 chunks of L
// samples, lane j owning chunk j.  The filters are linear, so lane j first runs its
// chunk from the zero state (f_j = its final state), the chunk-start states follow in
// one scan s_{j+1} = Phi s_j + f_j (s_0 = the state carried from the previous block,
// lane r computing component r), and each lane runs its chunk again from s_j, storing
// the raw band signals; the lane of the last chunk keeps its final state.
template <int NB>
__global__ void __launch_bounds__(32) k_rv_bands(RvShape sh, const float *__restrict__ in, unsigned char *state,
                                                 const double *__restrict__ phi_g, float *__restrict__ raw)
{
    constexpr int M = 8 * (NB - 1), MM = M > 0 ? M : 1;
    __shared__ double phi[MM * MM], T[33][MM];
    const int s = blockIdx.x, lane = threadIdx.x;
    const int N = sh.N, L = (N + 31) / 32;
    const int a = min(lane * L, N), e = min(a + L, N);
    double *zs = (double *)(state + (size_t)s * sh.bytes + sh.off_x);
    const float *x = in + (size_t)s * N;
    for (int q = lane; q < M * M; q += 32) phi[q] = phi_g[q];
    for (int r = lane; r < M; r += 32) T[0][r] = zs[r];
    double z[MM], y[NB];
    if (M > 0) {
#pragma unroll
        for (int r = 0; r < M; ++r) z[r] = 0.0;
        for (int n = a; n < e; ++n) tree_step<NB>(sh, z, (double)x[n], y);
#pragma unroll
        for (int r = 0; r < M; ++r) T[lane + 1][r] = z[r];
        __syncwarp();
        for (int j = 0; j < 31 && (j + 1) * L < N; ++j) {
            for (int r = lane; r < M; r += 32) {
                double acc = T[j + 1][r];
                for (int c = 0; c < M; ++c) acc = fma(phi[r * M + c], T[j][c], acc);
                T[j + 1][r] = acc;
            }
            __syncwarp();
        }
#pragma unroll
        for (int r = 0; r < M; ++r) z[r] = T[lane][r];
    }
    for (int n = a; n < e; ++n) {
        tree_step<NB>(sh, z, (double)x[n], y);
#pragma unroll
        for (int b = 0; b < NB; ++b) raw[((size_t)s * NB + b) * N + n] = (float)y[b];
    }
    if (a < e && e == N) {
#pragma unroll
        for (int r = 0; r < M; ++r) zs[r] = z[r];
    }
}

__device__ __forceinline__ int source_predelay(const RvShape &sh, const rp_reverb_params *prm, int s, int *status)
{
    int p = delay_samples(prm[(size_t)s * sh.B].predelay_s, sh.fs);
    if (p > sh.Pmax) {
        if (status) raise_error(status, RP_ERR_CAPACITY);
        p = sh.Pmax;
    }
    return p;
}

// the bands read at the predelay: this block's raw samples, or the ring of earlier ones
__global__ void k_rv_predelay(RvShape sh, const rp_reverb_params *prm, unsigned char *state,
                              const float *__restrict__ raw, float *__restrict__ bands, int *status)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)sh.S * sh.B * sh.N) return;
    const int n = (int)(id % sh.N);
    const long long sb = id / sh.N;
    const int s = (int)(sb / sh.B), b = (int)(sb - (long long)s * sh.B);
    const unsigned char *st = state + (size_t)s * sh.bytes;
    const long long n0 = *(const long long *)(st + sh.off_n0);
    const int p = source_predelay(sh, prm, s, n == 0 && b == 0 ? status : nullptr);
    const int L = sh.Pmax + 1;
    float v = 0.f;
    if (n >= p) v = raw[sb * sh.N + n - p];
    else if (n0 + n - p >= 0) v = ((const float *)(st + sh.off_pre))[(size_t)((n0 + n - p) % L) * sh.B + b];
    bands[id] = v;
}

// the last L raw samples go to the predelay ring (after every read of it)
__global__ void k_rv_predelay_store(RvShape sh, unsigned char *state, const float *__restrict__ raw)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)sh.S * sh.B * sh.N) return;
    const int n = (int)(id % sh.N);
    const long long sb = id / sh.N;
    const int s = (int)(sb / sh.B), b = (int)(sb - (long long)s * sh.B);
    const int L = sh.Pmax + 1;
    if (n < sh.N - L) return;
    unsigned char *st = state + (size_t)s * sh.bytes;
    const long long n0 = *(const long long *)(st + sh.off_n0);
    ((float *)(st + sh.off_pre))[(size_t)((n0 + n) % L) * sh.B + b] = raw[id];
}

// a block per (source, band): the N_comb combs one after another, each as its K-vector
// recurrence y[n] = comb_in x[n] + g J y[n - d] in chunks of d samples (the samples of
// a chunk depend only on the previous chunk, or on the comb's ring for the first, so a
// chunk's samples run in parallel); u accumulates the combs' sum, and the comb's last
// samples go to its ring
__global__ void __launch_bounds__(256) k_rv_combs(RvShape sh, const rp_reverberator *rev, unsigned char *state,
                                                  const float *__restrict__ bands, float *__restrict__ ys,
                                                  float *__restrict__ us, int *status)
{
    const int sb = blockIdx.x, s = sb / sh.B, b = sb - s * sh.B, K = sh.K, N = sh.N;
    unsigned char *st = state + (size_t)s * sh.bytes;
    const long long n0 = *(const long long *)(st + sh.off_n0);
    const rp_reverberator &R = rev[s];
    __shared__ float J[RP_MAX_SH][RP_MAX_SH], cin[RP_MAX_SH];
    const float *x = bands + (size_t)sb * N;
    float *y = ys + (size_t)sb * K * N, *u = us + (size_t)sb * K * N;  // [K][N]
    for (int i = 0; i < RP_N_COMB; ++i) {
        float *ring = (float *)(st + sh.off_comb) + ((size_t)b * RP_N_COMB + i) * sh.Dmax * K;
        int d = max(1, delay_samples(R.t_comb[i], sh.fs));
        if (d > sh.Dmax) {
            if (threadIdx.x == 0) raise_error(status, RP_ERR_CAPACITY);
            d = sh.Dmax;
        }
        const float g = (float)R.g_comb[i][b];
        for (int q = threadIdx.x; q < K * K; q += blockDim.x) J[q / K][q % K] = R.J[i][q / K][q % K];
        if (threadIdx.x < K) cin[threadIdx.x] = R.comb_in[i][threadIdx.x];
        __syncthreads();
        for (int c0 = 0; c0 < N; c0 += d) {
            const int c1 = min(c0 + d, N);
            for (int n = c0 + threadIdx.x; n < c1; n += blockDim.x) {
                const long long t = n0 + n;
                float yp[RP_MAX_SH];
#pragma unroll
                for (int k = 0; k < RP_MAX_SH; ++k) {
                    float v = 0.f;
                    if (k < K) {
                        if (n >= d) v = y[(size_t)k * N + n - d];
                        else if (t >= d) v = ring[(size_t)((t - d) % sh.Dmax) * K + k];
                    }
                    yp[k] = v;
                }
                const float xn = x[n];
#pragma unroll
                for (int k = 0; k < RP_MAX_SH; ++k) {
                    if (k >= K) break;
                    float fb = 0.f;
#pragma unroll
                    for (int kp = 0; kp < RP_MAX_SH; ++kp)
                        if (kp < K) fb = fmaf(J[k][kp], yp[kp], fb);
                    const float yn = fmaf(g, fb, cin[k] * xn);
                    y[(size_t)k * N + n] = yn;
                    u[(size_t)k * N + n] = i == 0 ? yn : u[(size_t)k * N + n] + yn;
                }
            }
            __syncthreads();  // the chunk is written before the next one reads it
        }
        for (int n = max(0, N - sh.Dmax) + threadIdx.x; n < N; n += blockDim.x)
            for (int k = 0; k < K; ++k) ring[(size_t)((n0 + n) % sh.Dmax) * K + k] = y[(size_t)k * N + n];
        __syncthreads();  // J, cin and y are reused by the next comb
    }
}

// a warp per (source, band, SH channel): the 4 all-pass stages over the combs' sum, in
// segments of AP_SEG samples held in shared memory with the stage's last d inputs and
// outputs in front (from its ring); within a stage, chunks of d samples run in
// parallel, v[n] = -a u[n] + u[n - d] + a v[n - d]; the stage's output is the next
// stage's input.  Each stage's ring keeps its last d inputs and outputs at (t mod d).
__global__ void k_rv_allpass(RvShape sh, unsigned char *state, float *__restrict__ us)
{
    extern __shared__ float ap_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * (blockDim.x >> 5) + warp;
    if (ch >= sh.S * sh.B * sh.K) return;  // warps are independent (no block barrier below)
    const int H = sh.ap_h, N = sh.N;
    float *bufA = ap_smem + (size_t)warp * 2 * (H + AP_SEG), *bufB = bufA + H + AP_SEG;
    const int sb = ch / sh.K, k = ch - sb * sh.K, s = sb / sh.B, b = sb - s * sh.B;
    unsigned char *st = state + (size_t)s * sh.bytes;
    const long long n0 = *(const long long *)(st + sh.off_n0);
    float *ring = (float *)(st + sh.off_ap) + ((size_t)b * sh.K + k) * sh.ap_len;  // the source's [B][K][ap_len]
    float *uc = us + (size_t)ch * N;
    const float ga = (float)AP_GAIN;
    for (int g0 = 0; g0 < N; g0 += AP_SEG) {
        const int L = min(AP_SEG, N - g0);
        const long long t0 = n0 + g0;
        float *vi = bufA, *vo = bufB;
        for (int n = lane; n < L; n += 32) vi[H + n] = uc[g0 + n];
        for (int a = 0; a < N_AP; ++a) {
            const int d = sh.ap_d[a];
            float *ri = ring + sh.ap_off[a], *ro = ri + d;
            for (int j = lane; j < d; j += 32) {
                const long long t = t0 - d + j;
                const int slot = t >= 0 ? (int)(t % d) : 0;
                vi[H - d + j] = t >= 0 ? ri[slot] : 0.f;
                vo[H - d + j] = t >= 0 ? ro[slot] : 0.f;
            }
            __syncwarp();
            for (int c0 = 0; c0 < L; c0 += d) {
                const int c1 = min(c0 + d, L);
                for (int n = c0 + lane; n < c1; n += 32)
                    vo[H + n] = fmaf(ga, vo[H + n - d], fmaf(-ga, vi[H + n], vi[H + n - d]));
                __syncwarp();
            }
            for (int j = lane; j < d; j += 32) {
                const long long t = t0 + L - d + j;
                if (t >= 0) {
                    const int slot = (int)(t % d);
                    ri[slot] = vi[H + L - d + j];
                    ro[slot] = vo[H + L - d + j];
                }
            }
            __syncwarp();
            float *tmp = vi;
            vi = vo;
            vo = tmp;
        }
        for (int n = lane; n < L; n += 32) uc[g0 + n] = vi[H + n];
        __syncwarp();
    }
}

__global__ void k_rv_out(RvShape sh, const rp_reverberator *rev, const rp_reverb_params *prm,
                         const float *__restrict__ v, float *__restrict__ out)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)sh.S * sh.N) return;
    const int s = (int)(id / sh.N), n = (int)(id - (long long)s * sh.N), K = sh.K;
    float q[RP_MAX_SH];
    for (int k = 0; k < RP_MAX_SH; ++k) q[k] = 0.f;
    for (int b = 0; b < sh.B; ++b) {
        const double gr = prm[(size_t)s * sh.B + b].g_reverb;
        const float g = isfinite(gr) ? (float)gr : 0.f;
        if (g == 0.f) continue;
        const float *vb = v + ((size_t)s * sh.B + b) * K * sh.N + n;
        float vk[RP_MAX_SH];
        for (int k = 0; k < K; ++k) vk[k] = vb[(size_t)k * sh.N];
        for (int k = 0; k < K; ++k) {
            float acc = 0.f;
            for (int kp = 0; kp < K; ++kp) acc = fmaf(rev[s].D[b][k][kp], vk[kp], acc);
            q[k] = fmaf(g, acc, q[k]);
        }
    }
    for (int k = 0; k < K; ++k) out[((size_t)s * K + k) * sh.N + n] = q[k];
}

__global__ void k_rv_advance(RvShape sh, unsigned char *state)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < sh.S) *(long long *)(state + (size_t)s * sh.bytes + sh.off_n0) += sh.N;
}

size_t ap_smem_per_warp(const RvShape &sh) { return sizeof(float) * 2 * (size_t)(sh.ap_h + AP_SEG); }

template <int NB>
void launch_bands(const RvShape &sh, const float *in, unsigned char *state, double *phi, float *raw, cudaStream_t st)
{
    const int L = (sh.N + 31) / 32;
    if (NB > 1) k_rv_phi<NB><<<1, 64, 0, st>>>(sh, L, phi);
    k_rv_bands<NB><<<sh.S, 32, 0, st>>>(sh, in, state, phi, raw);
}

void bands(const RvShape &sh, const float *in, unsigned char *state, double *phi, float *raw, cudaStream_t st)
{
    switch (sh.B) {
    case 1: launch_bands<1>(sh, in, state, phi, raw, st); break;
    case 2: launch_bands<2>(sh, in, state, phi, raw, st); break;
    case 3: launch_bands<3>(sh, in, state, phi, raw, st); break;
    case 4: launch_bands<4>(sh, in, state, phi, raw, st); break;
    case 5: launch_bands<5>(sh, in, state, phi, raw, st); break;
    case 6: launch_bands<6>(sh, in, state, phi, raw, st); break;
    case 7: launch_bands<7>(sh, in, state, phi, raw, st); break;
    default: launch_bands<8>(sh, in, state, phi, raw, st); break;
    }
}

bool make_shape(const rp_reverb_render_config *cfg, int S, int B, int K, int N, RvShape &sh)
{
    if (!cfg || S < 1 || B < 1 || B > RP_MAX_BANDS || K < 1 || K > RP_MAX_SH || N < 0 || !(cfg->sample_rate > 0.0) ||
        cfg->max_delay_samples < 1 || cfg->max_predelay_samples < 0)
        return false;
    const int n = (int)std::lround(std::sqrt((double)K)) - 1;
    if ((n + 1) * (n + 1) != K) return false;
    sh.S = S;
    sh.B = B;
    sh.K = K;
    sh.N = N;
    sh.fs = cfg->sample_rate;
    sh.Dmax = cfg->max_delay_samples;
    sh.Pmax = cfg->max_predelay_samples;
    double prev = 0.0;
    for (int x = 0; x < B - 1; ++x) {
        const double fc = cfg->crossover_hz[x];
        if (!(fc > prev) || !(fc < 0.5 * cfg->sample_rate)) return false;
        prev = fc;
        sh.lp[x] = butterworth2(fc, cfg->sample_rate, false);
        sh.hp[x] = butterworth2(fc, cfg->sample_rate, true);
    }
    int off = 0;
    for (int a = 0; a < N_AP; ++a) {
        sh.ap_d[a] = std::max(1, (int)std::floor(AP_MS[a] / 1000.0 * cfg->sample_rate + 0.5));
        sh.ap_off[a] = off;
        off += 2 * sh.ap_d[a];
    }
    sh.ap_len = off;
    sh.ap_h = sh.ap_d[0];
    if (ap_smem_per_warp(sh) > 48 * 1024) return false;  // sample rate above about 1 MHz
    layout(sh);
    return true;
}

}  // namespace
}  // namespace rp

extern "C" {

int rp_reverb_state_bytes(int32_t S, int32_t B, int32_t K, const rp_reverb_render_config *cfg, int64_t *bytes)
{
    RvShape sh;
    if (!bytes || !make_shape(cfg, S, B, K, 1, sh)) return RP_ERR_INVALID_ARG;
    *bytes = (int64_t)sh.bytes * S;
    return RP_OK;
}

int rp_reverb_render(rp_ctx *c, const rp_reverberator *rev, const rp_reverb_params *params, int32_t S, int32_t B,
                     int32_t K, const rp_reverb_render_config *cfg, const float *in, int32_t N, float *out, void *state)
{
    RvShape sh;
    if (!c || !rev || !params || !in || !out || !state || !make_shape(cfg, S, B, K, N, sh)) return RP_ERR_INVALID_ARG;
    if (N == 0) return RP_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return RP_ERR_CUDA;
    const size_t nb = sizeof(float) * (size_t)S * B * N, nk = sizeof(float) * (size_t)S * B * K * N;
    const size_t nphi = sizeof(double) * 64 * 64;
    for (auto q : {std::make_pair(&c->rv_raw, nb), std::make_pair(&c->rv_bands, nb), std::make_pair(&c->rv_comb, nk),
                   std::make_pair(&c->rv_ap, nk), std::make_pair(&c->rv_phi, nphi)}) {
        Buf &b = *q.first;
        if (b.bytes < q.second) {
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RP_ERR_CUDA;
            if (b.p) cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
            if (cudaMalloc(&b.p, q.second) != cudaSuccess) return RP_ERR_OOM;
            b.bytes = q.second;
        }
    }
    cudaStream_t st = c->stream;
    unsigned char *stt = (unsigned char *)state;
    float *raw = (float *)c->rv_raw.p, *bnd = (float *)c->rv_bands.p, *ys = (float *)c->rv_comb.p,
          *us = (float *)c->rv_ap.p;
    const long long nsbn = (long long)S * B * N;
    {
        ProfScope ps(c, "reverb_bands");
        bands(sh, in, stt, (double *)c->rv_phi.p, raw, st);
        k_rv_predelay<<<(unsigned)((nsbn + 255) / 256), 256, 0, st>>>(sh, params, stt, raw, bnd, c->d_status);
        k_rv_predelay_store<<<(unsigned)((nsbn + 255) / 256), 256, 0, st>>>(sh, stt, raw);
    }
    {
        ProfScope ps(c, "reverb_combs");
        k_rv_combs<<<S * B, 256, 0, st>>>(sh, rev, stt, bnd, ys, us, c->d_status);
    }
    {
        ProfScope ps(c, "reverb_allpass");
        const long long warps = (long long)S * B * K;
        const size_t smem = AP_WARPS * ap_smem_per_warp(sh);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k_rv_allpass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return RP_ERR_CUDA;
        k_rv_allpass<<<(unsigned)((warps + AP_WARPS - 1) / AP_WARPS), 32 * AP_WARPS, smem, st>>>(sh, stt, us);
    }
    {
        ProfScope ps(c, "reverb_out");
        const long long n = (long long)S * N;
        k_rv_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sh, rev, params, us, out);
    }
    k_rv_advance<<<(S + 63) / 64, 64, 0, st>>>(sh, stt);
    return cudaGetLastError() == cudaSuccess ? RP_OK : RP_ERR_CUDA;
}

}  // extern "C"
