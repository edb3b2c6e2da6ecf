// mlp_tc.cuh -- the learned estimator's fused forward pass on tcgen05 tensor cores
// (mlp_tc.cu), as called by mlp.cu.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rp {

constexpr int TC_MAX_N = 256;      // widest layer (TMEM columns of the accumulator)
constexpr int TC_MAX_LAYERS = 9;   // hidden layers + the output layer

// One launch: all layers for n samples.  Layer l: [n][kdim[l]] x Wt_l^T -> [n][ndim[l]],
// Wt_l stored [ndim][kdim] (K-major), bias[l] FP32.  Hidden layers: GELU; the output
// layer writes Y [n][ndim[last]] (FP32).  With Z (training), layer l's pre-activations
// and BF16 activations go to Z / Act + l act_stride, row stride ndim[l].
struct TcForwardParams {
    CUtensorMap xmap;                   // set by mlp_forward_tc
    CUtensorMap wmap[TC_MAX_LAYERS];    // Wt_l, boxes of 64 columns x ndim[l] rows
    const float *bias[TC_MAX_LAYERS];
    int kdim[TC_MAX_LAYERS];
    int ndim[TC_MAX_LAYERS];
    int nlayers;
    int n;
    float *Y;
    float *Z;
    __nv_bfloat16 *Act;
    long long act_stride;
    int *status;
};

bool mlp_tc_supported(int in_dim, int hidden, int layers, int out_dim);
bool tc_encode_map(CUtensorMap *map, const void *ptr, int rows, int cols, int box_rows);
// p.xmap must hold the input's map (tc_encode_map(X, n rows, in_dim columns, 128 rows))
cudaError_t mlp_forward_tc(const TcForwardParams &p, cudaStream_t st);
constexpr int TC_TILE_ROWS = 128;

}  // namespace rp
