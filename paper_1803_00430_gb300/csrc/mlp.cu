// mlp.cu -- learned reverberation-parameter estimator: a small MLP that maps a
// low-ray-count energy IR plus scene features to per-band decay times and
// direct-to-reverberant ratios, trained and run on the GPU with BF16 tensor-core
// GEMMs (FP32 accumulation), FP32 master weights and AdamW.
//
//   features   per band, the normalised energy-decay curve (Schroeder integral) of
//              X_b00(t) sampled at 63 equal steps of a window that ends where it
//              first falls below -40 dB, as log10(EDC + 1e-8), and the log of that
//              window's length in seconds; then log10 V (bounding box), log10 S
//              (triangle area), area-weighted mean absorption per band
//   network    in -> [GELU(W x + b)] x layers -> W x + b; weights W[in][out]
//   loss       masked mean squared error on standardised targets
//
// Forward pass: one fused launch on the tcgen05 tensor cores (mlp_tc.cu: TMA-staged
// operands, TMEM accumulators, bias / GELU epilogue, all layers per 128-sample tile)
// where the shape allows it (hidden width a multiple of 64 up to 256, output width a
// multiple of 16); otherwise, and for the backward pass, the GEMM below.
// GEMM: 64x64 block tile, 4 warps of 32x32, K-steps of 32 staged in shared memory
// (row stride 40 bf16: the fragment loads are bank-conflict free), mma.sync
// m16n8k16 BF16 -> FP32, epilogues fused: +bias, +bias then GELU (keeping the
// pre-activation for the backward pass), x GELU'(z) for the backward pass.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "handles.cuh"
#include "mlp_tc.cuh"

using namespace rp;

namespace {

typedef __nv_bfloat16 bf16;

constexpr int FEAT_BANDS = 8;
constexpr int FEAT_BINS = 64;
constexpr int FEAT_SCENE = 2 + FEAT_BANDS;
constexpr int FEAT_MIN = FEAT_BANDS * FEAT_BINS + FEAT_SCENE;  // 522
constexpr int FEAT_THREADS = 256;
constexpr int FEAT_MAX_T = 11264;       // T floats of decay curve in shared memory (44 KB)
constexpr double FEAT_FLOOR = 1e-4;     // -40 dB: end of each band's window
constexpr int FEAT_MIN_WINDOW = 4;      // bins

enum { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_GELU = 2, EPI_DGELU = 3 };

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.7071067811865476f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.7071067811865476f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M][N] = op(A)[M][K] x op(B)[K][N] with a fused epilogue.
//   A: AT ? stored [K][M] (lda) : stored [M][K]
//   B: BT ? stored [N][K] (ldb) : stored [K][N]
// blockIdx.z takes the K range [z kchunk, (z+1) kchunk) (split K, EPI_F32 only): its
// partial product goes to Cf + z M ldc and k_reduce_splits adds the partials.
template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, int kchunk, const bf16 *__restrict__ A, int lda,
                                              const bf16 *__restrict__ Bm, int ldb, float *__restrict__ Cf,
                                              bf16 *__restrict__ Cb, int ldc, const float *__restrict__ bias,
                                              const float *__restrict__ Zin, float *__restrict__ Zout)
{
    __shared__ __align__(16) bf16 As[64][40];
    __shared__ __align__(16) bf16 Bs[64][40];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t4 = lane & 3;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    if (EPI == EPI_F32) Cf += (size_t)blockIdx.z * M * ldc;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = kbeg; k0 < kend; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 128) {
            int mm, kk;
            if (!AT) {
                mm = e >> 5;
                kk = e & 31;
            } else {
                kk = e >> 6;
                mm = e & 63;
            }
            const int gm = m0 + mm, gk = k0 + kk;
            bf16 v = zero;
            if (gm < M && gk < kend) v = AT ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[mm][kk] = v;
        }
        for (int e = tid; e < 64 * 32; e += 128) {
            int nn, kk;
            if (BT) {
                nn = e >> 5;
                kk = e & 31;
            } else {
                kk = e >> 6;
                nn = e & 63;
            }
            const int gn = n0 + nn, gk = k0 + kk;
            bf16 v = zero;
            if (gn < N && gk < kend) v = BT ? Bm[(size_t)gn * ldb + gk] : Bm[(size_t)gk * ldb + gn];
            Bs[nn][kk] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < 32; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm * 32 + mt * 16 + g;
                af[mt][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + t4 * 2]);
                af[mt][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + t4 * 2]);
                af[mt][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + t4 * 2 + 8]);
                af[mt][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + t4 * 2 + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = wn * 32 + nt * 8 + g;
                bfr[nt][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][ks + t4 * 2]);
                bfr[nt][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][ks + t4 * 2 + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm * 32 + mt * 16 + g + (q >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + nt * 8 + t4 * 2 + (q & 1);
                if (m >= M || n >= N) continue;
                const size_t idx = (size_t)m * ldc + n;
                float v = acc[mt][nt][q];
                if (EPI == EPI_F32) {
                    Cf[idx] = v;
                } else if (EPI == EPI_BIAS_F32) {
                    Cf[idx] = v + bias[n];
                } else if (EPI == EPI_BIAS_GELU) {
                    v += bias[n];
                    Zout[idx] = v;
                    Cb[idx] = __float2bfloat16(gelu_f(v));
                } else {
                    Cb[idx] = __float2bfloat16(v * gelu_grad_f(Zin[idx]));
                }
            }
}

template <bool AT, bool BT, int EPI>
void gemm(cudaStream_t st, int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb, float *Cf, bf16 *Cb,
          int ldc, const float *bias = nullptr, const float *Zin = nullptr, float *Zout = nullptr)
{
    const dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<AT, BT, EPI><<<grid, 128, 0, st>>>(M, N, K, K, A, lda, B, ldb, Cf, Cb, ldc, bias, Zin, Zout);
}

constexpr int MAX_SPLIT = 16;    // K splits of a weight-gradient GEMM
constexpr int COLSUM_PARTS = 64;  // row chunks of a column sum

// out[i] = sum over z of part[z][i], z in order (deterministic)
__global__ void k_reduce_splits(long long count, int splits, const float *__restrict__ part, float *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * count + i];
        out[i] = s;
    }
}

// Weight gradient C[M][N] = A^T B with K = the batch: few output tiles and a long K,
// so K is split until the grid covers the SMs about twice.
void gemm_wgrad(cudaStream_t st, int num_sms, int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb,
                float *C, float *part)
{
    const dim3 tiles((N + 63) / 64, (M + 63) / 64);
    const int want = (2 * std::max(num_sms, 1) + (int)(tiles.x * tiles.y) - 1) / (int)(tiles.x * tiles.y);
    const int splits = std::max(1, std::min({MAX_SPLIT, want, (K + 255) / 256}));
    if (splits == 1) {
        k_gemm<true, false, EPI_F32><<<tiles, 128, 0, st>>>(M, N, K, K, A, lda, B, ldb, C, nullptr, N, nullptr,
                                                           nullptr, nullptr);
        return;
    }
    const int kchunk = ((K + splits - 1) / splits + 31) / 32 * 32;
    const int used = (K + kchunk - 1) / kchunk;
    k_gemm<true, false, EPI_F32><<<dim3(tiles.x, tiles.y, used), 128, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, part,
                                                                              nullptr, N, nullptr, nullptr, nullptr);
    const long long cnt = (long long)M * N;
    k_reduce_splits<<<(int)std::min<long long>((cnt + 255) / 256, 4096), 256, 0, st>>>(cnt, used, part, C);
}

__device__ __forceinline__ float to_f(bf16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f(float x) { return x; }

// stage 1: block (x, r) sums rows [r rows_per, (r+1) rows_per) of columns
// [32 x, 32 x + 32): thread (c, y) takes every 8th row, then the 8 partial sums of a
// column are added in order; stage 2 adds the row chunks in order (deterministic).
template <typename T>
__global__ void k_colsum_part(int M, int N, int rows_per, const T *__restrict__ X, float *__restrict__ part)
{
    __shared__ float sh[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * rows_per, r1 = min(M, r0 + rows_per);
    float s = 0.f;
    if (n < N)
        for (int m = r0 + threadIdx.y; m < r1; m += 8) s += to_f(X[(size_t)m * N + n]);
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += sh[y][threadIdx.x];
        part[(size_t)blockIdx.y * N + n] = t;
    }
}

__global__ void k_colsum_final(int N, int parts, const float *__restrict__ part, float *__restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int r = 0; r < parts; ++r) s += part[(size_t)r * N + n];
    out[n] = s;
}

// sums of the columns of an M x N matrix (bias gradients)
template <typename T>
void colsum(cudaStream_t st, int M, int N, const T *X, float *out, float *part)
{
    const int parts = std::max(1, std::min(COLSUM_PARTS, (M + 255) / 256));
    const int rows_per = (M + parts - 1) / parts;
    k_colsum_part<T><<<dim3((N + 31) / 32, parts), dim3(32, 8), 0, st>>>(M, N, rows_per, X, part);
    k_colsum_final<<<(N + 127) / 128, 128, 0, st>>>(N, parts, part, out);
}

__global__ void k_mask_sum(int count, const float *__restrict__ mask, float *__restrict__ out)
{
    float s = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) s += mask[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// dY = 2 mask (y - t) / max(1, sum mask); loss = sum mask (y - t)^2 / max(1, sum mask)
__global__ void k_loss_grad(int count, const float *__restrict__ Y, const float *__restrict__ Tg,
                            const float *__restrict__ mask, const float *__restrict__ msum, bf16 *__restrict__ dY,
                            float *__restrict__ loss)
{
    const float norm = fmaxf(1.0f, *msum);
    float l = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float r = Y[i] - Tg[i];
        l += mask[i] * r * r;
        dY[i] = __float2bfloat16(2.0f * mask[i] * r / norm);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(FULL, l, o);
    if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, l / norm);
}

// AdamW on the FP32 masters; refresh the BF16 copy of weight entries
__global__ void k_adamw(long long count, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                        float *__restrict__ v, float lr, float b1, float b2, float eps, float wd, float c1, float c2,
                        const long long *__restrict__ wmap, bf16 *__restrict__ pb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
        p[i] = pi;
        const long long j = wmap[i];
        if (j >= 0) pb[j] = __float2bfloat16(pi);
    }
}

__global__ void k_to_bf16_weights(long long count, const float *__restrict__ p, const long long *__restrict__ wmap,
                                  bf16 *__restrict__ pb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = wmap[i];
        if (j >= 0) pb[j] = __float2bfloat16(p[i]);
    }
}

// BF16 weights transposed for the tensor-core forward pass: wt[o][i] = w[i][o] of one layer
__global__ void k_transpose_w(int in, int out, const bf16 *__restrict__ w, bf16 *__restrict__ wt)
{
    __shared__ bf16 tile[32][33];
    const int i0 = blockIdx.x * 32, o0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = i0 + r, o = o0 + threadIdx.x;
        if (i < in && o < out) tile[r][threadIdx.x] = w[(size_t)i * out + o];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int o = o0 + r, i = i0 + threadIdx.x;
        if (i < in && o < out) wt[(size_t)o * in + i] = tile[threadIdx.x][r];
    }
}

// uniform(-a, a) initialisation of weights (a = sqrt(6 / (in + out))), zero biases
__global__ void k_init(long long count, float *__restrict__ p, const float *__restrict__ scale, unsigned long long seed)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const U4 r = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), 0x4d4c50u, 0u, (uint32_t)seed,
                                   (uint32_t)(seed >> 32));
        p[i] = scale[i] * (2.0f * u01(r.x) - 1.0f);
    }
}

// One block per (sample, band).  The decay curve D(t) = sum_{t' >= t} h(t') of the
// band's X_00 series, normalised by D(0), is a suffix sum: each thread sums a
// contiguous segment (FP64), a block scan gives the sum of all later segments, and a
// backward walk fills D for the segment.  D never increases (h >= 0), so the first
// bin below the floor is the number of bins at or above it.  Then 63 samples of D at
// t_end * i / 63 (i = 1..63, linear interpolation between bins) and ln(t_end / f_ir).
__global__ void __launch_bounds__(FEAT_THREADS)
    k_features(const float *__restrict__ H, int B, int K, int T, double ir_rate, const float *__restrict__ scene,
               int in_dim, float *__restrict__ X)
{
    extern __shared__ float edc[];
    __shared__ double part[FEAT_THREADS];
    __shared__ int above_sh;
    const int s = blockIdx.x / FEAT_BANDS, b = blockIdx.x % FEAT_BANDS, tid = threadIdx.x;
    float *x = X + (size_t)s * in_dim;
    if (b == 0) {
        if (tid < FEAT_SCENE) x[FEAT_BANDS * FEAT_BINS + tid] = scene[(size_t)s * FEAT_SCENE + tid];
        for (int f = FEAT_MIN + tid; f < in_dim; f += FEAT_THREADS) x[f] = 0.f;
    }
    const float *h = b < B ? H + ((size_t)s * B + b) * K * (size_t)T : nullptr;
    const int L = (T + FEAT_THREADS - 1) / FEAT_THREADS;
    const int j0 = min(T, tid * L), j1 = min(T, j0 + L);
    double seg = 0.0;
    if (h)
        for (int j = j0; j < j1; ++j) seg += (double)h[j];
    part[tid] = seg;
    if (tid == 0) above_sh = 0;
    __syncthreads();
    for (int off = 1; off < FEAT_THREADS; off <<= 1) {  // inclusive suffix scan
        const double v = tid + off < FEAT_THREADS ? part[tid + off] : 0.0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    const double tot = part[0];
    double run = tid + 1 < FEAT_THREADS ? part[tid + 1] : 0.0;
    int above = 0;
    for (int j = j1 - 1; j >= j0; --j) {
        if (h) run += (double)h[j];
        const double r = tot > 0.0 ? run / tot : 0.0;
        edc[j] = (float)r;
        above += r >= FEAT_FLOOR;
    }
    atomicAdd(&above_sh, above);
    __syncthreads();
    const double t_end = (double)max(above_sh, FEAT_MIN_WINDOW);
    if (tid < FEAT_BINS - 1) {
        const double pos = fmin(t_end * (tid + 1) / (FEAT_BINS - 1), T - 1.001);
        const int i0 = (int)floor(pos), i1 = min(i0 + 1, T - 1);
        const double w = pos - i0;
        x[b * FEAT_BINS + tid] = (float)log10((double)edc[i0] * (1.0 - w) + (double)edc[i1] * w + 1e-8);
    } else if (tid == FEAT_BINS - 1) {
        x[b * FEAT_BINS + tid] = (float)log(t_end / ir_rate);
    }
}

__global__ void k_standardize(long long count, int in_dim, const float *__restrict__ X, const float *__restrict__ mean,
                              const float *__restrict__ istd, bf16 *__restrict__ Xb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % in_dim);
        Xb[i] = __float2bfloat16((X[i] - mean[f]) * istd[f]);
    }
}

__global__ void k_destandardize(long long count, int out_dim, float *__restrict__ Y, const float *__restrict__ mean,
                                const float *__restrict__ std)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % out_dim);
        Y[i] = Y[i] * std[f] + mean[f];
    }
}

// triangle area and area-weighted absorption of a scene (scene features)
__global__ void k_scene_sums(const float4 *__restrict__ tris, int nt, const float *__restrict__ alpha, int B,
                             double *__restrict__ out /* [1 + B] */)
{
    double area = 0.0, aw[MAXB];
    for (int b = 0; b < MAXB; ++b) aw[b] = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const float4 a = tris[3 * t], b4 = tris[3 * t + 1], c = tris[3 * t + 2];
        const float3 n = cross(xyz(b4) - xyz(a), xyz(c) - xyz(a));
        const double ar = 0.5 * sqrt((double)dot(n, n));
        area += ar;
        const int m = __float_as_int(a.w);
        for (int b = 0; b < B; ++b) aw[b] += ar * (double)alpha[m * B + b];
    }
    for (int o = 16; o > 0; o >>= 1) {
        area += __shfl_xor_sync(FULL, area, o);
        for (int b = 0; b < MAXB; ++b) aw[b] += __shfl_xor_sync(FULL, aw[b], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, area);
        for (int b = 0; b < B; ++b) atomicAdd(out + 1 + b, aw[b]);
    }
}

long long blocks_for(long long n) { return std::max(1ll, std::min((n + 255) / 256, 4096ll)); }

}  // namespace

struct rp_mlp {
    rp_ctx *ctx = nullptr;
    rp_mlp_config cfg;
    long long nparams = 0, nweights = 0;
    std::vector<long long> w_off, b_off, wb_off;  // master offsets of W and b, bf16 offsets of W
    std::vector<int> in_of, out_of;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 masters, gradients, moments
    bf16 *pb = nullptr;                                           // BF16 weights
    bf16 *wt = nullptr;                                           // BF16 weights transposed, [out][in] per layer
    bool use_tc = false;                                          // forward pass on the tcgen05 tensor cores
    TcForwardParams tc;                                           // its weight tensor maps and layer shapes
    const void *tc_x = nullptr;                                   // input whose map tc.xmap holds
    int tc_n = 0;
    long long *wmap = nullptr;                                    // master index -> bf16 index or -1
    float *in_mean = nullptr, *in_istd = nullptr, *out_mean = nullptr, *out_std = nullptr;
    float *Z = nullptr, *Y = nullptr, *scratch = nullptr;         // workspace for max_batch
    bf16 *Act = nullptr, *dA = nullptr, *dB = nullptr, *dY = nullptr;
    float *part = nullptr, *cpart = nullptr;  // split-K and column-sum partials
    int step = 0;
};

namespace {

int mrc(cudaError_t e)
{
    if (e == cudaSuccess) return RP_OK;
    if (e == cudaErrorMemoryAllocation) return RP_ERR_OOM;
    return RP_ERR_CUDA;
}

#define CKM(x)                                   \
    do {                                         \
        const cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) return mrc(e_);   \
    } while (0)

// the transposed BF16 weights of every layer, from the BF16 weights
void refresh_transposed(rp_mlp *mp, cudaStream_t st)
{
    if (!mp->use_tc) return;
    for (size_t l = 0; l < mp->in_of.size(); ++l) {
        const int in = mp->in_of[l], out = mp->out_of[l];
        k_transpose_w<<<dim3((in + 31) / 32, (out + 31) / 32), dim3(32, 8), 0, st>>>(in, out, mp->pb + mp->wb_off[l],
                                                                                    mp->wt + mp->wb_off[l]);
    }
}

// forward pass; with `keep` (training) it keeps the pre-activations Z[l] (f32) and the
// activations Act[l] (bf16) for the backward pass
void forward(rp_mlp *mp, const bf16 *X, int n, cudaStream_t st, bool keep = true)
{
    const rp_mlp_config &c = mp->cfg;
    const int L = c.layers, H = c.hidden;
    if (mp->use_tc) {
        TcForwardParams p = mp->tc;
        p.n = n;
        p.Y = mp->Y;
        p.Z = keep ? mp->Z : nullptr;
        p.Act = keep ? mp->Act : nullptr;
        p.act_stride = (long long)c.max_batch * H;
        p.status = mp->ctx->d_status;
        bool ok = true;
        if (X != mp->tc_x || n != mp->tc_n) {  // the input's tensor map, re-made when it changes
            ok = tc_encode_map(&mp->tc.xmap, X, n, c.in_dim, TC_TILE_ROWS);
            mp->tc_x = ok ? X : nullptr;
            mp->tc_n = ok ? n : 0;
            p.xmap = mp->tc.xmap;
        }
        if (ok) {
            ProfScope ps(mp->ctx, "mlp_forward_tc");
            if (mlp_forward_tc(p, st) == cudaSuccess) return;
        }
        mp->use_tc = false;  // the maps could not be made for this input: the GEMM path from now on
    }
    const bf16 *in = X;
    int width = c.in_dim;
    ProfScope ps(mp->ctx, "mlp_forward_gemm");
    for (int l = 0; l < L; ++l) {
        float *Zl = mp->Z + (size_t)l * c.max_batch * H;
        bf16 *Al = mp->Act + (size_t)l * c.max_batch * H;
        gemm<false, false, EPI_BIAS_GELU>(st, n, H, width, in, width, mp->pb + mp->wb_off[l], H, nullptr, Al, H,
                                          mp->p + mp->b_off[l], nullptr, Zl);
        in = Al;
        width = H;
    }
    gemm<false, false, EPI_BIAS_F32>(st, n, c.out_dim, width, in, width, mp->pb + mp->wb_off[L], c.out_dim, mp->Y,
                                     nullptr, c.out_dim, mp->p + mp->b_off[L]);
}

// loss and gradients of the masked MSE into mp->g; loss (device float) or NULL
void backward(rp_mlp *mp, const bf16 *X, const float *Tg, const float *mask, int n, float *loss, cudaStream_t st)
{
    const rp_mlp_config &c = mp->cfg;
    const int L = c.layers, H = c.hidden, O = c.out_dim;
    float *msum = mp->scratch;
    cudaMemsetAsync(msum, 0, sizeof(float), st);
    if (loss) cudaMemsetAsync(loss, 0, sizeof(float), st);
    const long long cnt = (long long)n * O;
    k_mask_sum<<<(int)blocks_for(cnt), 256, 0, st>>>((int)cnt, mask, msum);
    k_loss_grad<<<(int)blocks_for(cnt), 256, 0, st>>>((int)cnt, mp->Y, Tg, mask, msum, mp->dY, loss);
    // output layer
    const bf16 *a_last = L > 0 ? mp->Act + (size_t)(L - 1) * c.max_batch * H : X;
    const int w_last = L > 0 ? H : c.in_dim;
    const int sms = mp->ctx->num_sms;
    gemm_wgrad(st, sms, w_last, O, n, a_last, w_last, mp->dY, O, mp->g + mp->w_off[L], mp->part);
    colsum<bf16>(st, n, O, mp->dY, mp->g + mp->b_off[L], mp->cpart);
    const bf16 *delta = mp->dY;
    int dw = O;
    bf16 *bufs[2] = {mp->dA, mp->dB};
    for (int l = L - 1; l >= 0; --l) {
        // delta_l = (delta_{l+1} W_{l+1}^T) * gelu'(z_l)
        bf16 *dl = bufs[l & 1];
        gemm<false, true, EPI_DGELU>(st, n, H, dw, delta, dw, mp->pb + mp->wb_off[l + 1], dw, nullptr, dl, H, nullptr,
                                     mp->Z + (size_t)l * c.max_batch * H);
        const bf16 *a_in = l > 0 ? mp->Act + (size_t)(l - 1) * c.max_batch * H : X;
        const int w_in = l > 0 ? H : c.in_dim;
        gemm_wgrad(st, sms, w_in, H, n, a_in, w_in, dl, H, mp->g + mp->w_off[l], mp->part);
        colsum<bf16>(st, n, H, dl, mp->g + mp->b_off[l], mp->cpart);
        delta = dl;
        dw = H;
    }
}

}  // namespace

extern "C" {

int rp_mlp_create(rp_ctx *ctx, const rp_mlp_config *cfg, rp_mlp **out)
{
    if (!ctx || !cfg || !out) return RP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->in_dim < FEAT_MIN || cfg->in_dim % 8 || cfg->hidden < 8 || cfg->hidden % 8 || cfg->layers < 1 ||
        cfg->layers > 8 || cfg->out_dim < 1 || cfg->max_batch < 1)
        return RP_ERR_INVALID_ARG;
    CKM(cudaSetDevice(ctx->device));
    rp_mlp *mp = new (std::nothrow) rp_mlp();
    if (!mp) return RP_ERR_OOM;
    mp->ctx = ctx;
    mp->cfg = *cfg;
    const int L = cfg->layers;
    long long off = 0, boff = 0;
    for (int l = 0; l <= L; ++l) {
        const int in = l == 0 ? cfg->in_dim : cfg->hidden, outd = l == L ? cfg->out_dim : cfg->hidden;
        mp->in_of.push_back(in);
        mp->out_of.push_back(outd);
        mp->w_off.push_back(off);
        mp->wb_off.push_back(boff);
        off += (long long)in * outd;
        boff += (long long)in * outd;
        mp->b_off.push_back(off);
        off += outd;
    }
    mp->nparams = off;
    mp->nweights = boff;
    std::vector<long long> wmap(off, -1);
    std::vector<float> scale(off, 0.f);
    for (int l = 0; l <= L; ++l) {
        const long long cnt = (long long)mp->in_of[l] * mp->out_of[l];
        const float a = std::sqrt(6.0f / (float)(mp->in_of[l] + mp->out_of[l]));
        for (long long i = 0; i < cnt; ++i) {
            wmap[mp->w_off[l] + i] = mp->wb_off[l] + i;
            scale[mp->w_off[l] + i] = a;
        }
    }
    const size_t act = (size_t)cfg->max_batch * cfg->hidden;
    float *d_scale = nullptr;
    cudaError_t e;
    int rc = RP_OK;
    std::vector<float> ones(cfg->in_dim, 1.f), zeros(std::max(cfg->in_dim, cfg->out_dim), 0.f),
        oones(cfg->out_dim, 1.f);
    if ((e = cudaMalloc(&mp->p, sizeof(float) * off)) || (e = cudaMalloc(&mp->g, sizeof(float) * off)) ||
        (e = cudaMalloc(&mp->m, sizeof(float) * off)) || (e = cudaMalloc(&mp->v, sizeof(float) * off)) ||
        (e = cudaMalloc(&mp->pb, sizeof(bf16) * boff)) || (e = cudaMalloc(&mp->wmap, sizeof(long long) * off)) ||
        (e = cudaMalloc(&d_scale, sizeof(float) * off)) ||
        (e = cudaMalloc(&mp->in_mean, sizeof(float) * cfg->in_dim)) ||
        (e = cudaMalloc(&mp->in_istd, sizeof(float) * cfg->in_dim)) ||
        (e = cudaMalloc(&mp->out_mean, sizeof(float) * cfg->out_dim)) ||
        (e = cudaMalloc(&mp->out_std, sizeof(float) * cfg->out_dim)) ||
        (e = cudaMalloc(&mp->Z, sizeof(float) * act * L)) || (e = cudaMalloc(&mp->Act, sizeof(bf16) * act * L)) ||
        (e = cudaMalloc(&mp->dA, sizeof(bf16) * act)) || (e = cudaMalloc(&mp->dB, sizeof(bf16) * act)) ||
        (e = cudaMalloc(&mp->Y, sizeof(float) * (size_t)cfg->max_batch * cfg->out_dim)) ||
        (e = cudaMalloc(&mp->dY, sizeof(bf16) * (size_t)cfg->max_batch * cfg->out_dim)) ||
        (e = cudaMalloc(&mp->part, sizeof(float) * MAX_SPLIT * (size_t)std::max(cfg->in_dim, cfg->hidden) *
                                       std::max(cfg->hidden, cfg->out_dim))) ||
        (e = cudaMalloc(&mp->cpart, sizeof(float) * COLSUM_PARTS * (size_t)std::max(cfg->hidden, cfg->out_dim))) ||
        (e = cudaMalloc(&mp->scratch, sizeof(float) * 16))) {
        rc = mrc(e);
        goto fail;
    }
    if ((e = cudaMemcpy(mp->wmap, wmap.data(), sizeof(long long) * off, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_scale, scale.data(), sizeof(float) * off, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(mp->in_mean, zeros.data(), sizeof(float) * cfg->in_dim, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(mp->in_istd, ones.data(), sizeof(float) * cfg->in_dim, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(mp->out_mean, zeros.data(), sizeof(float) * cfg->out_dim, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(mp->out_std, oones.data(), sizeof(float) * cfg->out_dim, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(mp->m, 0, sizeof(float) * off)) || (e = cudaMemset(mp->v, 0, sizeof(float) * off))) {
        rc = mrc(e);
        goto fail;
    }
    if (!(cfg->flags & RP_MLP_FLAG_LEGACY_GEMM) && mlp_tc_supported(cfg->in_dim, cfg->hidden, L, cfg->out_dim)) {
        if ((e = cudaMalloc(&mp->wt, sizeof(bf16) * boff))) {
            rc = mrc(e);
            goto fail;
        }
        mp->use_tc = true;
        mp->tc.nlayers = L + 1;
        for (int l = 0; l <= L && mp->use_tc; ++l) {
            mp->tc.kdim[l] = mp->in_of[l];
            mp->tc.ndim[l] = mp->out_of[l];
            mp->tc.bias[l] = mp->p + mp->b_off[l];
            mp->use_tc = tc_encode_map(&mp->tc.wmap[l], mp->wt + mp->wb_off[l], mp->out_of[l], mp->in_of[l],
                                       mp->out_of[l]);
        }
    }
    k_init<<<(int)blocks_for(off), 256>>>(off, mp->p, d_scale, cfg->seed);
    k_to_bf16_weights<<<(int)blocks_for(off), 256>>>(off, mp->p, mp->wmap, mp->pb);
    refresh_transposed(mp, 0);
    if ((e = cudaDeviceSynchronize())) {
        rc = mrc(e);
        goto fail;
    }
    cudaFree(d_scale);
    *out = mp;
    return RP_OK;
fail:
    cudaFree(d_scale);
    rp_mlp_destroy(mp);
    return rc;
}

int rp_mlp_destroy(rp_mlp *mp)
{
    if (!mp) return RP_ERR_INVALID_ARG;
    cudaSetDevice(mp->ctx->device);
    cudaStreamSynchronize(mp->ctx->stream);
    for (void *q : {(void *)mp->p, (void *)mp->g, (void *)mp->m, (void *)mp->v, (void *)mp->pb, (void *)mp->wmap,
                    (void *)mp->in_mean, (void *)mp->in_istd, (void *)mp->out_mean, (void *)mp->out_std, (void *)mp->wt,
                    (void *)mp->Z, (void *)mp->Act, (void *)mp->dA, (void *)mp->dB, (void *)mp->Y, (void *)mp->dY,
                    (void *)mp->part, (void *)mp->cpart, (void *)mp->scratch})
        cudaFree(q);
    delete mp;
    return RP_OK;
}

int rp_mlp_param_count(const rp_mlp *mp, int64_t *count)
{
    if (!mp || !count) return RP_ERR_INVALID_ARG;
    *count = mp->nparams;
    return RP_OK;
}

int rp_mlp_get_params(rp_mlp *mp, float *params)
{
    if (!mp || !params) return RP_ERR_INVALID_ARG;
    CKM(cudaMemcpyAsync(params, mp->p, sizeof(float) * mp->nparams, cudaMemcpyDeviceToDevice, mp->ctx->stream));
    return RP_OK;
}

int rp_mlp_set_params(rp_mlp *mp, const float *params)
{
    if (!mp || !params) return RP_ERR_INVALID_ARG;
    cudaStream_t st = mp->ctx->stream;
    CKM(cudaMemcpyAsync(mp->p, params, sizeof(float) * mp->nparams, cudaMemcpyDeviceToDevice, st));
    k_to_bf16_weights<<<(int)blocks_for(mp->nparams), 256, 0, st>>>(mp->nparams, mp->p, mp->wmap, mp->pb);
    refresh_transposed(mp, st);
    return mrc(cudaGetLastError());
}

int rp_mlp_get_adam_state(rp_mlp *mp, float *m, float *v, int32_t *step)
{
    if (!mp || !m || !v || !step) return RP_ERR_INVALID_ARG;
    CKM(cudaMemcpyAsync(m, mp->m, sizeof(float) * mp->nparams, cudaMemcpyDeviceToDevice, mp->ctx->stream));
    CKM(cudaMemcpyAsync(v, mp->v, sizeof(float) * mp->nparams, cudaMemcpyDeviceToDevice, mp->ctx->stream));
    *step = mp->step;
    return RP_OK;
}

int rp_mlp_set_adam_state(rp_mlp *mp, const float *m, const float *v, int32_t step)
{
    if (!mp || !m || !v || step < 0) return RP_ERR_INVALID_ARG;
    CKM(cudaMemcpyAsync(mp->m, m, sizeof(float) * mp->nparams, cudaMemcpyDeviceToDevice, mp->ctx->stream));
    CKM(cudaMemcpyAsync(mp->v, v, sizeof(float) * mp->nparams, cudaMemcpyDeviceToDevice, mp->ctx->stream));
    mp->step = step;
    return RP_OK;
}

int rp_mlp_set_normalization(rp_mlp *mp, const float *in_mean, const float *in_std, const float *out_mean,
                             const float *out_std)
{
    if (!mp || !in_mean || !in_std || !out_mean || !out_std) return RP_ERR_INVALID_ARG;
    const int D = mp->cfg.in_dim, O = mp->cfg.out_dim;
    std::vector<float> istd(D);
    for (int i = 0; i < D; ++i) istd[i] = in_std[i] > 0.f ? 1.0f / in_std[i] : 1.0f;
    cudaStream_t st = mp->ctx->stream;
    CKM(cudaMemcpyAsync(mp->in_mean, in_mean, sizeof(float) * D, cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(mp->in_istd, istd.data(), sizeof(float) * D, cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(mp->out_mean, out_mean, sizeof(float) * O, cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(mp->out_std, out_std, sizeof(float) * O, cudaMemcpyHostToDevice, st));
    CKM(cudaStreamSynchronize(st));  // istd is a stack buffer
    return RP_OK;
}

int rp_scene_features(rp_scene *sc, float *out)
{
    if (!sc || !out) return RP_ERR_INVALID_ARG;
    rp_ctx *c = sc->ctx;
    CKM(cudaSetDevice(c->device));
    double *d = nullptr;
    CKM(cudaMalloc(&d, sizeof(double) * (1 + MAXB)));
    cudaMemsetAsync(d, 0, sizeof(double) * (1 + MAXB), c->stream);
    k_scene_sums<<<(int)std::min(1024ll, std::max(1ll, (long long)(sc->num_tris + 255) / 256)), 256, 0, c->stream>>>(
        sc->tris, sc->num_tris, sc->alpha, sc->B, d);
    double h[1 + MAXB];
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    CKM(e);
    double vol = 1.0;
    for (int k = 0; k < 3; ++k) vol *= std::max(1e-9, (double)sc->hi[k] - (double)sc->lo[k]);
    out[0] = (float)std::log10(vol);
    out[1] = (float)std::log10(std::max(h[0], 1e-12));
    for (int b = 0; b < FEAT_BANDS; ++b) out[2 + b] = b < sc->B && h[0] > 0 ? (float)(h[1 + b] / h[0]) : 0.f;
    return RP_OK;
}

int rp_mlp_features(rp_ctx *c, const float *H, int32_t S, int32_t B, int32_t K, int32_t T, float ir_rate_hz,
                    const float *scene_feats, int32_t in_dim, float *X)
{
    if (!c || !H || !scene_feats || !X || S < 1 || B < 1 || B > FEAT_BANDS || K < 1 || T < FEAT_MIN_WINDOW ||
        in_dim < FEAT_MIN || !(ir_rate_hz > 0.f) || !std::isfinite(ir_rate_hz))
        return RP_ERR_INVALID_ARG;
    if (T > FEAT_MAX_T) return RP_ERR_TOO_LARGE;
    CKM(cudaSetDevice(c->device));
    k_features<<<(unsigned)S * FEAT_BANDS, FEAT_THREADS, sizeof(float) * T, c->stream>>>(
        H, B, K, T, (double)ir_rate_hz, scene_feats, in_dim, X);
    return mrc(cudaGetLastError());
}

int rp_mlp_prepare(rp_mlp *mp, const float *X, int32_t n, void *Xb)
{
    if (!mp || !X || !Xb || n < 1) return RP_ERR_INVALID_ARG;
    const long long cnt = (long long)n * mp->cfg.in_dim;
    k_standardize<<<(int)blocks_for(cnt), 256, 0, mp->ctx->stream>>>(cnt, mp->cfg.in_dim, X, mp->in_mean, mp->in_istd,
                                                                     (bf16 *)Xb);
    return mrc(cudaGetLastError());
}

int rp_mlp_forward(rp_mlp *mp, const void *Xb, int32_t n, float *Y, int32_t destandardize)
{
    if (!mp || !Xb || !Y || n < 1 || n > mp->cfg.max_batch) return RP_ERR_INVALID_ARG;
    cudaStream_t st = mp->ctx->stream;
    forward(mp, (const bf16 *)Xb, n, st, false);
    const long long cnt = (long long)n * mp->cfg.out_dim;
    CKM(cudaMemcpyAsync(Y, mp->Y, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, st));
    if (destandardize)
        k_destandardize<<<(int)blocks_for(cnt), 256, 0, st>>>(cnt, mp->cfg.out_dim, Y, mp->out_mean, mp->out_std);
    return mrc(cudaGetLastError());
}

int rp_mlp_loss_grad(rp_mlp *mp, const void *Xb, const float *Tg, const float *mask, int32_t n, float *loss,
                     float *grad)
{
    if (!mp || !Xb || !Tg || !mask || n < 1 || n > mp->cfg.max_batch) return RP_ERR_INVALID_ARG;
    cudaStream_t st = mp->ctx->stream;
    forward(mp, (const bf16 *)Xb, n, st);
    backward(mp, (const bf16 *)Xb, Tg, mask, n, loss, st);
    if (grad) CKM(cudaMemcpyAsync(grad, mp->g, sizeof(float) * mp->nparams, cudaMemcpyDeviceToDevice, st));
    return mrc(cudaGetLastError());
}

int rp_mlp_train_step(rp_mlp *mp, const void *Xb, const float *Tg, const float *mask, int32_t n, float lr,
                      float weight_decay, float *loss)
{
    if (!mp || !Xb || !Tg || !mask || n < 1 || n > mp->cfg.max_batch || !(lr >= 0.f) || !(weight_decay >= 0.f))
        return RP_ERR_INVALID_ARG;
    cudaStream_t st = mp->ctx->stream;
    forward(mp, (const bf16 *)Xb, n, st);
    backward(mp, (const bf16 *)Xb, Tg, mask, n, loss, st);
    mp->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - std::pow(b1, (float)mp->step), c2 = 1.0f - std::pow(b2, (float)mp->step);
    k_adamw<<<(int)blocks_for(mp->nparams), 256, 0, st>>>(mp->nparams, mp->p, mp->g, mp->m, mp->v, lr, b1, b2, eps,
                                                           weight_decay, c1, c2, mp->wmap, mp->pb);
    refresh_transposed(mp, st);
    return mrc(cudaGetLastError());
}

}  // extern "C"
