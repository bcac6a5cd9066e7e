// sampler.cuh -- the fetch of Algorithm 1 ("val <- cube[loc]") for each storage.
//
// Positions arrive as 32.32 fixed-point coordinates (ray.cuh).  Trilinear
// interpolation is written by hand in FP32 from point loads: the texture unit's
// linear filter uses low-precision fixed-point weights and cannot meet the
// accuracy target.  Indices clamp to the edge voxel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "ray.cuh"

namespace shw {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ float lerp(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

// Tensor-product interpolation of the 8 corner values c[z][y][x].
__device__ __forceinline__ float trilerp(float c000, float c001, float c010, float c011, float c100, float c101,
                                         float c110, float c111, float fx, float fy, float fz)
{
    const float c00 = lerp(c000, c001, fx), c01 = lerp(c010, c011, fx);
    const float c10 = lerp(c100, c101, fx), c11 = lerp(c110, c111, fx);
    return lerp(lerp(c00, c01, fy), lerp(c10, c11, fy), fz);
}

// Linear float32 cube [nz][ny][nx].  Idx: int for < 2^31 voxels, long long beyond.
template <typename Idx>
struct SamplerF32 {
    const float *__restrict__ v;
    int nx, ny, nz;
    Idx sy, sz;  // strides of y and z in elements

    __device__ __forceinline__ float nearest(long long X, long long Y, long long Z) const
    {
        const int x = clampi(fx_round(X), 0, nx - 1), y = clampi(fx_round(Y), 0, ny - 1),
                  z = clampi(fx_round(Z), 0, nz - 1);
        return __ldg(v + ((Idx)z * sz + (Idx)y * sy + x));
    }

    // corner values c[z][y][x] of the cell with base (ix, iy, iz), each in [-1, n-1]
    __device__ __forceinline__ void corners(int ix, int iy, int iz, float c[8]) const
    {
        const int x0 = max(ix, 0), y0 = max(iy, 0), z0 = max(iz, 0);
        const int dx = min(ix + 1, nx - 1) - x0;
        const Idx dy = (Idx)(min(iy + 1, ny - 1) - y0) * sy;
        const Idx dz = (Idx)(min(iz + 1, nz - 1) - z0) * sz;
        const float *p00 = v + ((Idx)z0 * sz + (Idx)y0 * sy + x0);
        const float *p01 = p00 + dy, *p10 = p00 + dz, *p11 = p10 + dy;
        c[0] = __ldg(p00);
        c[1] = __ldg(p00 + dx);
        c[2] = __ldg(p01);
        c[3] = __ldg(p01 + dx);
        c[4] = __ldg(p10);
        c[5] = __ldg(p10 + dx);
        c[6] = __ldg(p11);
        c[7] = __ldg(p11 + dx);
    }

    __device__ __forceinline__ float trilinear(long long X, long long Y, long long Z) const
    {
        const int ix = clampi(fx_cell(X), -1, nx - 1), iy = clampi(fx_cell(Y), -1, ny - 1),
                  iz = clampi(fx_cell(Z), -1, nz - 1);
        const float fx = fx_frac(X), fy = fx_frac(Y), fz = fx_frac(Z);
        const int x0 = max(ix, 0), y0 = max(iy, 0), z0 = max(iz, 0);
        const int dx = min(ix + 1, nx - 1) - x0;
        const Idx dy = (Idx)(min(iy + 1, ny - 1) - y0) * sy;
        const Idx dz = (Idx)(min(iz + 1, nz - 1) - z0) * sz;
        const float *p00 = v + ((Idx)z0 * sz + (Idx)y0 * sy + x0);
        const float *p01 = p00 + dy, *p10 = p00 + dz, *p11 = p10 + dy;
        return trilerp(__ldg(p00), __ldg(p00 + dx), __ldg(p01), __ldg(p01 + dx), __ldg(p10), __ldg(p10 + dx),
                       __ldg(p11), __ldg(p11 + dx), fx, fy, fz);
    }
};

// 1: reuse the 8 corners of the cell a ray is in until it leaves that cell; 0: no reuse
#ifndef SHW_CELL_CACHE
#define SHW_CELL_CACHE 1
#endif

// The corners c[a + 2b + 4c] (a, b, c = x, y, z offsets) of the last interpolation cell
// a ray visited.  Consecutive samples 1/2 voxel apart often stay in one cell and then
// need no loads at all.
struct CellCache {
    int ix = -4, iy = -4, iz = -4;  // no cell yet: valid cells start at -1
    float c[8];
};

template <class S>
__device__ __forceinline__ float trilinear_cached(const S &s, long long X, long long Y, long long Z, CellCache &cc)
{
    const int ix = clampi(fx_cell(X), -1, s.nx - 1), iy = clampi(fx_cell(Y), -1, s.ny - 1),
              iz = clampi(fx_cell(Z), -1, s.nz - 1);
    if (ix != cc.ix || iy != cc.iy || iz != cc.iz) {
        s.corners(ix, iy, iz, cc.c);
        cc.ix = ix;
        cc.iy = iy;
        cc.iz = iz;
    }
    return trilerp(cc.c[0], cc.c[1], cc.c[2], cc.c[3], cc.c[4], cc.c[5], cc.c[6], cc.c[7], fx_frac(X), fx_frac(Y),
                   fx_frac(Z));
}

template <typename T>
__device__ __forceinline__ float to_f32(unsigned short raw);
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(unsigned short raw)
{
    return __uint_as_float(((unsigned)raw) << 16);
}
template <>
__device__ __forceinline__ float to_f32<__half>(unsigned short raw)
{
    return __half2float(__ushort_as_half(raw));
}

// 32^3 bricks with a 1-voxel replicated apron, stored as 34^3 16-bit values
// (layout documented with shw_pack_bricks).  The apron makes the 8 corners of
// every cell live in one brick, at fixed offsets from the cell's base.
template <typename T>
struct SamplerBrick {
    const unsigned short *__restrict__ v;
    int nx, ny, nz;
    int nbx, nby;

    static constexpr int S = kBrickStored;

    __device__ __forceinline__ const unsigned short *cell(int ix, int iy, int iz) const
    {
        // ix in [-1, n-1]: brick of max(ix, 0), local index ix - 32 b + 1 in [0, 32]
        const int bx = max(ix, 0) >> 5, by = max(iy, 0) >> 5, bz = max(iz, 0) >> 5;
        const int lx = ix - (bx << 5) + 1, ly = iy - (by << 5) + 1, lz = iz - (bz << 5) + 1;
        const long long brick = ((long long)bz * nby + by) * nbx + bx;
        return v + (brick * kBrickElems + (lz * S + ly) * S + lx);
    }

    __device__ __forceinline__ float nearest(long long X, long long Y, long long Z) const
    {
        const int x = clampi(fx_round(X), 0, nx - 1), y = clampi(fx_round(Y), 0, ny - 1),
                  z = clampi(fx_round(Z), 0, nz - 1);
        const int bx = x >> 5, by = y >> 5, bz = z >> 5;
        const long long brick = ((long long)bz * nby + by) * nbx + bx;
        const unsigned short *p = v + (brick * kBrickElems + (((z & 31) + 1) * S + ((y & 31) + 1)) * S + (x & 31) + 1);
        return to_f32<T>(__ldg(p));
    }

    __device__ __forceinline__ void corners(int ix, int iy, int iz, float c[8]) const
    {
        const unsigned short *p = cell(ix, iy, iz);
        c[0] = to_f32<T>(__ldg(p));
        c[1] = to_f32<T>(__ldg(p + 1));
        c[2] = to_f32<T>(__ldg(p + S));
        c[3] = to_f32<T>(__ldg(p + S + 1));
        c[4] = to_f32<T>(__ldg(p + S * S));
        c[5] = to_f32<T>(__ldg(p + S * S + 1));
        c[6] = to_f32<T>(__ldg(p + S * S + S));
        c[7] = to_f32<T>(__ldg(p + S * S + S + 1));
    }

    __device__ __forceinline__ float trilinear(long long X, long long Y, long long Z) const
    {
        const int ix = clampi(fx_cell(X), -1, nx - 1), iy = clampi(fx_cell(Y), -1, ny - 1),
                  iz = clampi(fx_cell(Z), -1, nz - 1);
        const float fx = fx_frac(X), fy = fx_frac(Y), fz = fx_frac(Z);
        const unsigned short *p = cell(ix, iy, iz);
        return trilerp(to_f32<T>(__ldg(p)), to_f32<T>(__ldg(p + 1)), to_f32<T>(__ldg(p + S)),
                       to_f32<T>(__ldg(p + S + 1)), to_f32<T>(__ldg(p + S * S)), to_f32<T>(__ldg(p + S * S + 1)),
                       to_f32<T>(__ldg(p + S * S + S)), to_f32<T>(__ldg(p + S * S + S + 1)), fx, fy, fz);
    }
};

}  // namespace shw
