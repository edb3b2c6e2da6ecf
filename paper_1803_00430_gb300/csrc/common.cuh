// common.cuh -- device helpers shared by the CUDA kernels of the library:
// Philox4x32-10, real spherical harmonics in Cartesian form, vector math,
// warp-aggregated appends and the device status word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rpr.h"

namespace rp {

constexpr int MAXB = RP_MAX_BANDS;
constexpr int MAXK = RP_MAX_SH;
constexpr float PI_F = 3.14159265358979323846f;
constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Device status: the first error wins; later ones are dropped.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void raise_error(int *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// Bounds checks of the RP_CHECKED build: the kernels test every reflection, record,
// key, cell and histogram index they compute (node and triangle indices are tested
// in every build) before using it; a violation records RP_ERR_BOUNDS and the access
// is skipped.  Without RP_CHECKED the test compiles to `true`.
__device__ __forceinline__ bool checked_index(unsigned long long i, unsigned long long n, int *status)
{
    if (i < n) return true;
    raise_error(status, RP_ERR_BOUNDS);
    return false;
}
#ifdef RP_CHECKED
#define RP_IN_RANGE(i, n, status) ::rp::checked_index((unsigned long long)(i), (unsigned long long)(n), (status))
#else
#define RP_IN_RANGE(i, n, status) true
#endif

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies with the published multipliers, key bumped by the Weyl constants.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// uniform in [0,1) from the top 24 bits; exact in float
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// float3 helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 mk3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 xyz(float4 v) { return mk3(v.x, v.y, v.z); }

// Primary direction of ray `rid`: uniform on the sphere from the bounce-0 draws,
// z = 1 - 2 u0, phi = 2 pi u1.
__device__ __forceinline__ float3 primary_direction(uint32_t rid, uint32_t scene_id, uint32_t k0,
                                                    uint32_t k1)
{
    const U4 r = philox4x32_10(rid, scene_id, 0u, 0u, k0, k1);
    const float z = 1.0f - 2.0f * u01(r.x);
    const float rad = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float s, c;
    sincospif(2.0f * u01(r.y), &s, &c);
    return mk3(rad * c, rad * s, z);
}

// ---------------------------------------------------------------------------
// Real orthonormal spherical harmonics with the Condon-Shortley phase, ACN index
// k = l*l + l + m, as polynomials of a unit vector (orders 0..3).  Under this sign
// convention the first-order coefficients of a single direction d are
// (-c d.y, c d.z, -c d.x), so (-X11, -X1-1, X10) points along d.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sh_eval(int order, float x, float y, float z, float *Y)
{
    Y[0] = 0.28209479177387814f;
    if (order < 1) return;
    const float c1 = 0.4886025119029199f;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (order < 2) return;
    const float c2a = 1.0925484305920792f, c20 = 0.31539156525252005f, c22 = 0.5462742152960396f;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c20 * (3.0f * z * z - 1.0f);
    Y[7] = -c2a * x * z;
    Y[8] = c22 * (x * x - y * y);
    if (order < 3) return;
    const float c33 = 0.5900435899266435f, c32a = 2.890611442640554f, c32b = 1.445305721320277f;
    const float c31 = 0.4570457994644658f, c30 = 0.3731763325901154f;
    const float z2 = z * z;
    Y[9] = -c33 * y * (3.0f * x * x - y * y);
    Y[10] = c32a * x * y * z;
    Y[11] = -c31 * y * (5.0f * z2 - 1.0f);
    Y[12] = c30 * z * (5.0f * z2 - 3.0f);
    Y[13] = -c31 * x * (5.0f * z2 - 1.0f);
    Y[14] = c32b * z * (x * x - y * y);
    Y[15] = -c33 * x * (x * x - 3.0f * y * y);
}

// ---------------------------------------------------------------------------
// Warp-aggregated append: one atomic per group of converged lanes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_append(unsigned long long *counter)
{
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
}

// 64-bit FNV-1a over the four little-endian bytes of v
__device__ __forceinline__ uint64_t fnv_u32(uint64_t h, uint32_t v)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h ^= (v >> (8 * i)) & 0xffu;
        h *= 0x100000001b3ull;
    }
    return h;
}

constexpr uint64_t FNV_OFFSET = 0xcbf29ce484222325ull;

}  // namespace rp
