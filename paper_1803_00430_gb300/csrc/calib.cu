// calib.cu -- measured throughput of the FP32 pipes that bound BVH traversal, for the
// rooflines of the tracing kernels (the paper has no counterpart).
//
// Two kernels of independent dependency chains, enough warps per SM to hide the
// latency of each instruction:
//   k_fma_chain     eight chains of x = fma(x, a, b) per thread: FP32 fused multiply-add
//                   instructions per second (the FMA pipe; 2 flops each);
//   k_minmax_chain  eight chains of x = min(max(x, a), b) per thread: FP32 min / max
//                   instructions per second (the ALU pipe, where the slab tests' min,
//                   max and compares issue).  Alternating min and max keeps every
//                   operation one instruction.
// Each is timed with CUDA events on the context stream, best of five launches.
#include "handles.cuh"

namespace rp {
namespace {

constexpr int CAL_THREADS = 256;
constexpr int CAL_ITERS = 4096;
constexpr int CAL_CHAINS = 8;

__global__ void __launch_bounds__(CAL_THREADS) k_fma_chain(float a, float b, float *out)
{
    float x[CAL_CHAINS];
#pragma unroll
    for (int c = 0; c < CAL_CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < CAL_ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < CAL_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CAL_CHAINS; ++c) s += x[c];
    if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live; never true for the inputs used
}

__global__ void __launch_bounds__(CAL_THREADS) k_minmax_chain(float a, float b, float *out)
{
    float x[CAL_CHAINS];
#pragma unroll
    for (int c = 0; c < CAL_CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
    float lo = a, hi = b;
    for (int i = 0; i < CAL_ITERS; ++i) {
        lo += 1.0f;  // loop-variant bounds: the chains cannot be folded
        hi -= 1.0f;
#pragma unroll
        for (int c = 0; c < CAL_CHAINS; ++c) x[c] = fminf(fmaxf(x[c], lo), hi);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CAL_CHAINS; ++c) s += x[c];
    if (s == 1234.5f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace rp

using namespace rp;

extern "C" int rp_measure_pipe_peaks(rp_ctx *c, double *fma_per_s, double *minmax_per_s)
{
    if (!c || !fma_per_s || !minmax_per_s) return RP_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return RP_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chain, CAL_THREADS, 0);
    const int blocks = c->num_sms * (per_sm > 0 ? per_sm : 1) * 4;
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) return RP_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double ops = (double)blocks * CAL_THREADS * CAL_ITERS * CAL_CHAINS;
    double best[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2; ++kind) {
        // the min/max kernel makes two instructions per chain step
        const double n = kind == 0 ? ops : 2.0 * ops;
        for (int rep = 0; rep < 6; ++rep) {
            cudaEventRecord(e0, c->stream);
            if (kind == 0) k_fma_chain<<<blocks, CAL_THREADS, 0, c->stream>>>(1.0000001f, 1e-7f, out);
            else k_minmax_chain<<<blocks, CAL_THREADS, 0, c->stream>>>(-1e30f, 1e30f, out);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms > 0.f) best[kind] = std::max(best[kind], n / (ms * 1e-3));  // the first warms up
        }
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return RP_ERR_CUDA;
    *fma_per_s = best[0];
    *minmax_per_s = best[1];
    return RP_OK;
}
