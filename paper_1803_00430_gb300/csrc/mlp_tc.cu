// mlp_tc.cu -- the learned estimator's forward pass on the 5th-generation tensor cores:
// every layer of the MLP for a tile of 128 samples in one CTA, with tcgen05.mma BF16
// x BF16 -> FP32 accumulators in tensor memory (TMEM), operands staged by TMA in the
// 128-byte swizzled K-major layout, and the bias / GELU epilogue fused.
//
// CTA of 18 warps, one 128-sample tile:
//   warp 16 (one lane)  producer: TMA of the weight K-chunks of every layer (and of the
//                       input tile's K-chunks for layer 0) into a three-stage ring;
//   warp 17 (one lane)  MMA issuer: per 64-wide K-chunk four tcgen05.mma of K = 16
//                       (M = 128, N = layer width), accumulating in TMEM; commits free
//                       the ring stages and, after a layer's last chunk, signal the
//                       epilogue;
//   warps 0-15          epilogue: tcgen05.ld of the accumulators (warp w reads TMEM
//                       lanes 32 (w mod 4) .. + 31, i.e. those samples, and a quarter
//                       of the columns), + bias (staged in shared memory at the start),
//                       GELU (erf form) for hidden layers, written back
//                       to shared memory in the swizzled layout as the next layer's A
//                       operand (and, when training, the pre-activations Z and the
//                       BF16 activations to global memory), or the output Y.
// The activation tile never leaves the SM between layers; weights come from L2.
//
// Every wait on an mbarrier is bounded (about 2 s of SM clock); a wait that runs out
// records RP_ERR_TIMEOUT, raises an abort flag that the other roles poll, and the CTA
// drains what it issued before it frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "handles.cuh"
#include "mlp_tc.cuh"

namespace rp {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TC_M = 128;           // samples per CTA (TMEM lanes)
constexpr int TC_KC = 64;           // K elements per chunk: 128 bytes of BF16, one swizzle row
constexpr int TC_NST = 3;           // ring stages
constexpr int TC_EPI_WARPS = 16;   // four per TMEM lane quarter, a quarter of the columns each
constexpr int TC_THREADS = (TC_EPI_WARPS + 2) * 32;
constexpr uint32_t TC_A_BYTES = TC_M * 128;         // one K-chunk of the 128-sample tile
constexpr uint32_t TC_B_BYTES = TC_MAX_N * 128;     // one K-chunk of the widest weight tile
constexpr uint32_t TC_ACT_BYTES = (TC_MAX_N / TC_KC) * TC_A_BYTES;
constexpr uint32_t TC_BIAS_BYTES = TC_MAX_LAYERS * TC_MAX_N * 4;
constexpr uint32_t TC_SMEM =
    1024 /* alignment */ + TC_ACT_BYTES + TC_NST * (TC_A_BYTES + TC_B_BYTES) + TC_BIAS_BYTES + 256;
constexpr long long TC_WAIT_CYCLES = 4000000000ll;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// true once the phase with parity `parity` has completed; the thread may sleep in the
// wait for up to about 20 microseconds (it wakes when the phase completes)
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "n"(20000)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with parity `parity` of `bar`; false when it ran out (the
// timeout is recorded and the abort flag raised) or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status)
{
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            raise_error(status, RP_ERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major BF16 operand in the 128-byte swizzled
// layout: rows of 128 bytes (64 K-elements), 8-row groups 1024 bytes apart (stride
// byte offset), the leading byte offset unused; descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (tmem_wait_ld completes it)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// GELU (erf form) with erf from Abramowitz & Stegun, Handbook of Mathematical Functions,
// formula 7.1.26 (after Hastings): erf(x) = 1 - (a1 t + ... + a5 t^5) exp(-x^2),
// t = 1 / (1 + p x) for x >= 0, |error| <= 1.5e-7, odd in x -- far below the BF16
// rounding of the activation it feeds; fast reciprocal and exponential.
__device__ __forceinline__ float gelu_tc(float z)
{
    const float x = fabsf(z) * 0.7071067811865476f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    const float erf_abs = fmaf(-poly * t, __expf(-x * x), 1.0f);
    const float e = copysignf(erf_abs, z);
    return 0.5f * z * (1.0f + e);
}

// Packed FP32 pairs (sm_100 and later): one instruction for two lanes' worth of FP32
// arithmetic, round to nearest, the same results as the scalar operations.
__device__ __forceinline__ unsigned long long pk2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// GELU of two values at once: the same formula as gelu_tc (Abramowitz & Stegun 7.1.26
// for erf), its multiplications and additions on packed pairs
__device__ __forceinline__ void gelu_tc2(float z0, float z1, float &g0, float &g1)
{
    const float c = 0.7071067811865476f;
    const unsigned long long Z = pk2(z0, z1);
    const unsigned long long X = pk2(fabsf(z0) * c, fabsf(z1) * c);
    float d0, d1;
    upk2(fma2(X, pk2(0.3275911f, 0.3275911f), pk2(1.0f, 1.0f)), d0, d1);
    const unsigned long long T = pk2(__fdividef(1.0f, d0), __fdividef(1.0f, d1));
    unsigned long long poly = fma2(T, pk2(1.061405429f, 1.061405429f), pk2(-1.453152027f, -1.453152027f));
    poly = fma2(T, poly, pk2(1.421413741f, 1.421413741f));
    poly = fma2(T, poly, pk2(-0.284496736f, -0.284496736f));
    poly = fma2(T, poly, pk2(0.254829592f, 0.254829592f));
    const unsigned long long PT = mul2(poly, T);
    float y0, y1;
    upk2(mul2(X, X), y0, y1);
    const unsigned long long E = pk2(__expf(-y0), __expf(-y1));
    float m0, m1;  // 1 - erf(|x|) ... as poly t exp(-x^2), then erf with the sign of z
    upk2(fma2(PT, E, pk2(-1.0f, -1.0f)), m0, m1);  // -(erf |x|)
    const unsigned long long EZ = pk2(copysignf(-m0, z0), copysignf(-m1, z1));
    upk2(mul2(mul2(Z, pk2(0.5f, 0.5f)), add2(EZ, pk2(1.0f, 1.0f))), g0, g1);
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_forward_tc(const __grid_constant__ TcForwardParams p)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *act = base;                                       // next layer's A operand
    unsigned char *stage_a = base + TC_ACT_BYTES;                    // [TC_NST][TC_A_BYTES]
    unsigned char *stage_b = stage_a + TC_NST * TC_A_BYTES;          // [TC_NST][TC_B_BYTES]
    float *sbias = (float *)(stage_b + TC_NST * TC_B_BYTES);         // [TC_MAX_LAYERS][TC_MAX_N]
    uint64_t *bars = (uint64_t *)(sbias + TC_MAX_LAYERS * TC_MAX_N);
    uint64_t *full = bars, *empty = bars + TC_NST, *accum_full = bars + 2 * TC_NST, *act_ready = accum_full + 1,
             *drain = act_ready + 1;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * TC_M;
    for (int l = 0; l < p.nlayers; ++l)
        for (int c = threadIdx.x; c < p.ndim[l]; c += blockDim.x) sbias[l * TC_MAX_N + c] = __ldg(p.bias[l] + c);
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum_full, 1);
        mbar_init(act_ready, TC_EPI_WARPS * 32);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // the whole warp allocates the accumulator columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)TC_MAX_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nl = p.nlayers;

    if (warp == TC_EPI_WARPS) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int l = 0; l < nl && ok; ++l) {
                const int nk = (p.kdim[l] + TC_KC - 1) / TC_KC;
                const uint32_t bbytes = (uint32_t)p.ndim[l] * 128u;
                for (int kc = 0; kc < nk && ok; ++kc, ++it) {
                    const int s = it % TC_NST;
                    if (it >= TC_NST) ok = mbar_wait(&empty[s], ((it / TC_NST) - 1) & 1, abort_flag, p.status);
                    if (!ok) break;
                    mbar_arrive_expect_tx(&full[s], bbytes + (l == 0 ? TC_A_BYTES : 0u));
                    tma_load_2d(stage_b + s * TC_B_BYTES, &p.wmap[l], &full[s], kc * TC_KC, 0);
                    if (l == 0) tma_load_2d(stage_a + s * TC_A_BYTES, &p.xmap, &full[s], kc * TC_KC, row0);
                }
            }
            // the copies this lane issued complete before the CTA leaves: wait for the
            // ring's last phases (bounded; stages that were never armed are skipped)
            for (int j = (it > TC_NST ? it - TC_NST : 0); j < it; ++j) {
                const long long t0 = clock64();
                while (!mbar_test(&full[j % TC_NST], (j / TC_NST) & 1) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == TC_EPI_WARPS + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            bool issued = false;
            for (int l = 0; l < nl && ok; ++l) {
                if (l > 0) {
                    ok = mbar_wait(act_ready, (l - 1) & 1, abort_flag, p.status);
                    if (!ok) break;
                    tc_fence_after();
                }
                const int nk = (p.kdim[l] + TC_KC - 1) / TC_KC;
                const uint32_t idesc = idesc_bf16(TC_M, p.ndim[l]);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % TC_NST;
                    ok = mbar_wait(&full[s], (it / TC_NST) & 1, abort_flag, p.status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_base =
                        l == 0 ? smem_u32(stage_a + s * TC_A_BYTES) : smem_u32(act + kc * TC_A_BYTES);
                    const uint32_t b_base = smem_u32(stage_b + s * TC_B_BYTES);
#pragma unroll
                    for (int k = 0; k < TC_KC / 16; ++k) {
                        // K = 16 BF16 = 32 bytes further along the swizzled 128-byte rows
                        umma_bf16(tmem, sdesc_sw128(a_base + 32u * k), sdesc_sw128(b_base + 32u * k), idesc,
                                  (kc > 0 || k > 0) ? 1u : 0u);
                    }
                    issued = true;
                    umma_commit(&empty[s]);  // the stage is free once these MMAs have read it
                }
                if (ok) umma_commit(accum_full);
            }
            if (issued) {  // every MMA this lane issued has completed before TMEM is freed
                umma_commit(drain);
                const long long t0 = clock64();
                while (!mbar_test(drain, 0) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 0-7 ----------------
        const int q = warp & 3;                 // TMEM lane quarter = the samples 32 q .. 32 q + 31
        const int part = warp >> 2;             // the quarter of the columns this warp takes
        const int r = q * 32 + lane;            // sample within the tile
        const int row = row0 + r;
        for (int l = 0; l < nl; ++l) {
            // the warp goes on together (the TMEM loads below are warp-collective)
            if (!__all_sync(0xffffffffu, mbar_wait(accum_full, l & 1, abort_flag, p.status))) break;
            tc_fence_after();
            const int N = p.ndim[l];
            const bool last = l == nl - 1;
            const int cw = N / 4;  // columns per quarter (a multiple of 16 for hidden layers)
            const float *bias = sbias + l * TC_MAX_N;
            // 32 columns per round: two TMEM loads, one wait
            for (int c00 = part * cw; c00 < (part + 1) * cw; c00 += 32) {
                uint32_t rr[2][16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c00, rr[0]);
                if (c00 + 16 < (part + 1) * cw) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c00 + 16), rr[1]);
                tmem_wait_ld();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c0 = c00 + 16 * h;
                    if (c0 >= (part + 1) * cw) break;
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(rr[h][i]);
                    const int cn = min(16, (part + 1) * cw - c0);
                    if (last) {
                        if (row < p.n) {
                            float *y = p.Y + (size_t)row * p.ndim[l] + c0;
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (i < cn) y[i] = v[i] + bias[c0 + i];
                        }
                        continue;
                    }
                    uint32_t packed[8];
                    if (cn == 16) {  // every column of the chunk (hidden layers: always)
                        const float2 *b2 = reinterpret_cast<const float2 *>(bias + c0);
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            const float2 bb = b2[i / 2];
                            float z0, z1, g0, g1;
                            upk2(add2(pk2(v[i], v[i + 1]), pk2(bb.x, bb.y)), z0, z1);
                            v[i] = z0;
                            v[i + 1] = z1;
                            gelu_tc2(z0, z1, g0, g1);
                            const __nv_bfloat162 a2 = __floats2bfloat162_rn(g0, g1);
                            packed[i / 2] = *reinterpret_cast<const uint32_t *>(&a2);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            const float z0 = v[i] + (i < cn ? bias[c0 + i] : 0.f);
                            const float z1 = v[i + 1] + (i + 1 < cn ? bias[c0 + i + 1] : 0.f);
                            v[i] = z0;
                            v[i + 1] = z1;
                            const __nv_bfloat162 a2 = __floats2bfloat162_rn(gelu_tc(z0), gelu_tc(z1));
                            packed[i / 2] = *reinterpret_cast<const uint32_t *>(&a2);
                        }
                    }
                    // next layer's A operand: K-chunk c0 / 64, row r, 16-byte units j, j + 1
                    // of the 128-byte row, swizzled (unit index XOR row mod 8)
                    unsigned char *rowp = act + (c0 / TC_KC) * TC_A_BYTES + r * 128;
                    const int j = (c0 % TC_KC) / 8;
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (u * 8 < cn) {
                            uint4 w4 =
                                make_uint4(packed[4 * u], packed[4 * u + 1], packed[4 * u + 2], packed[4 * u + 3]);
                            *reinterpret_cast<uint4 *>(rowp + (((j + u) ^ (r & 7)) * 16)) = w4;
                        }
                    }
                    if (p.Z && row < p.n) {  // training keeps Z and the BF16 activations
                        float *zrow = p.Z + (size_t)l * p.act_stride + (size_t)row * N + c0;
                        bf16 *arow = p.Act + (size_t)l * p.act_stride + (size_t)row * N + c0;
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (i < cn) zrow[i] = v[i];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (2 * i < cn) reinterpret_cast<uint32_t *>(arow)[i] = packed[i];
                    }
                }
            }
            if (last) break;
            // the activations become the next layer's operand: visible to the tensor cores,
            // this thread's TMEM reads complete, then its arrival (the MMA issuer waits for
            // all of the epilogue's threads; no thread waits on another here)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            mbar_arrive(act_ready);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TC_MAX_N)
                     : "memory");
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)f;
    });
    return fn;
}

}  // namespace

bool mlp_tc_supported(int in_dim, int hidden, int layers, int out_dim)
{
    return in_dim % 8 == 0 && hidden % TC_KC == 0 && hidden >= TC_KC && hidden <= TC_MAX_N && out_dim % 16 == 0 &&
           out_dim >= 16 && out_dim <= TC_MAX_N && layers + 1 <= TC_MAX_LAYERS;
}

// 2-D BF16 tensor map of a row-major [rows][cols] matrix with 64-column x box_rows
// boxes in the 128-byte swizzle; elements outside the matrix read as zero.
bool tc_encode_map(CUtensorMap *map, const void *ptr, int rows, int cols, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc || ((uintptr_t)ptr & 15u) || (cols * 2) % 16) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_KC, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t mlp_forward_tc(const TcForwardParams &p, cudaStream_t st)
{
    // the kernel's shared memory beyond 48 KB is opted into once per device
    static std::mutex mu;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 0 || dev >= 64 || !attr_done[dev]) {
            e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) attr_done[dev] = true;
        }
    }
    const int grid = (p.n + TC_M - 1) / TC_M;
    k_mlp_forward_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(p);
    return cudaGetLastError();
}

}  // namespace rp
