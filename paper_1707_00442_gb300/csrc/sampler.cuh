// sampler.cuh -- the fetch of Algorithm 1 ("val <- cube[loc]") for each storage.
//
// Positions arrive as 32.32 fixed-point coordinates (ray.cuh).  Trilinear
// interpolation is written by hand in FP32 from point loads: the texture unit's
// linear filter uses low-precision fixed-point weights and cannot meet the
// accuracy target.  Indices clamp to the edge voxel.  Every accessor has a
// clamp-free form (CLAMP = false) for samples whose cell is known to lie in
// [0, n-2] on every axis, where both corners of each axis are inside the cube.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "ray.cuh"

namespace shw {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ float lerp(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

// two lerps at once with packed FP32x2 arithmetic (same rounding as two scalar lerps)
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float t)
{
    const float2 d = __fadd2_rn(b, make_float2(-a.x, -a.y));
    return __ffma2_rn(make_float2(t, t), d, a);
}

// Corners of one cell, c[a + 2b + 4c] with a, b, c the x, y, z offsets.
// Tensor-product interpolation: x first, then y, then z.  The lerps go in pairs across the
// two z planes, so each level's packed result is the next level's operand as it stands.
__device__ __forceinline__ float trilerp(const float c[8], float fx, float fy, float fz)
{
    const float2 y0 = lerp2(make_float2(c[0], c[4]), make_float2(c[1], c[5]), fx);  // row y0 of planes z0, z1
    const float2 y1 = lerp2(make_float2(c[2], c[6]), make_float2(c[3], c[7]), fx);  // row y1 of planes z0, z1
    const float2 z = lerp2(y0, y1, fy);                                              // planes z0, z1
    return lerp(z.x, z.y, fz);
}

template <bool CLAMP>
__device__ __forceinline__ int cell_of(long long p, int n)
{
    return CLAMP ? clampi(fx_cell(p), -1, n - 1) : fx_cell(p);
}

// Bounds-checked builds (SHW_CHECKED): the contract of an unclamped accessor -- the base of a
// cell with both corners inside the cube ([0, n-2] per axis), a voxel inside it, a brick cell
// in [-1, n-1] -- is checked; a violating index is recorded and clamped into its range.
// Normal builds: no code.
__device__ __forceinline__ void check_range(int &i, int lo, int hi)
{
    if constexpr (kChecked) {
        const bool ok = i >= lo && i <= hi;
        SHW_CHECK(ok);
        if (!ok) i = max(min(i, hi), lo);
    }
}
__device__ __forceinline__ void check_cell(int &ix, int &iy, int &iz, int nx, int ny, int nz)
{
    check_range(ix, 0, nx - 2);
    check_range(iy, 0, ny - 2);
    check_range(iz, 0, nz - 2);
}
__device__ __forceinline__ void check_voxel(int &x, int &y, int &z, int nx, int ny, int nz)
{
    check_range(x, 0, nx - 1);
    check_range(y, 0, ny - 1);
    check_range(z, 0, nz - 1);
}

// Linear float32 cube [nz][ny][nx].  Idx: int for < 2^31 voxels, long long beyond.
template <typename Idx>
struct SamplerF32 {
    static constexpr bool kLinearF32 = true;
    static constexpr bool kPair = false;
    const float *__restrict__ v;
    int nx, ny, nz;
    Idx sy, sz;  // strides of y and z in elements

    template <bool CLAMP = true>
    __device__ __forceinline__ float nearest(long long X, long long Y, long long Z) const
    {
        int x = fx_round(X), y = fx_round(Y), z = fx_round(Z);
        if (CLAMP) {
            x = clampi(x, 0, nx - 1);
            y = clampi(y, 0, ny - 1);
            z = clampi(z, 0, nz - 1);
        } else {
            check_voxel(x, y, z, nx, ny, nz);
        }
        return __ldg(v + ((Idx)z * sz + (Idx)y * sy + x));
    }

    // corners of the cell with base (ix, iy, iz); CLAMP: each index in [-1, n-1]
    template <bool CLAMP = true>
    __device__ __forceinline__ void corners(int ix, int iy, int iz, float c[8]) const
    {
        if (!CLAMP) check_cell(ix, iy, iz, nx, ny, nz);
        int x0 = ix, y0 = iy, z0 = iz, dx = 1;
        Idx dy = sy, dz = sz;
        if (CLAMP) {
            x0 = max(ix, 0);
            y0 = max(iy, 0);
            z0 = max(iz, 0);
            dx = min(ix + 1, nx - 1) - x0;
            dy = (Idx)(min(iy + 1, ny - 1) - y0) * sy;
            dz = (Idx)(min(iz + 1, nz - 1) - z0) * sz;
        }
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
        float c[8];
        corners<true>(cell_of<true>(X, nx), cell_of<true>(Y, ny), cell_of<true>(Z, nz), c);
        return trilerp(c, fx_frac(X), fx_frac(Y), fx_frac(Z));
    }
};

template <typename T>
__device__ __forceinline__ float to_f32(unsigned short raw);
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(unsigned short raw)
{
    // the bfloat16 bits are the float's high half: raw * 2^16 (an integer multiply, on the
    // FMA pipe, instead of a shift on the busier integer ALU pipe; same bits)
    return __uint_as_float((unsigned)raw * 65536u);
}
template <>
__device__ __forceinline__ float to_f32<__half>(unsigned short raw)
{
    return __half2float(__ushort_as_half(raw));
}

// E^3 bricks (E = 32 for shw_pack_bricks; batch plans that pack their own bricks also
// use 16) with a 1-voxel replicated apron, stored as (E+2)^3 16-bit values (layout
// documented with shw_pack_bricks).  The apron makes the 8 corners of every cell live in
// one brick, at fixed offsets from the cell's base.
// Idx: int when the brick buffer holds < 2^31 elements (cheaper address arithmetic), else long long.
template <typename T, typename Idx = long long, int E = kBrick>
struct SamplerBrick {
    static_assert(E == 16 || E == 32, "brick edge 16 or 32");
    static constexpr bool kLinearF32 = false;
    static constexpr bool kPair = false;
    const unsigned short *__restrict__ v;
    int nx, ny, nz;
    int nbx, nby;

    static constexpr int kShift = E == 16 ? 4 : 5;
    static constexpr int S = E + 2 * SHW_BRICK_APRON;
    static constexpr int kElems = S * S * S;

    __device__ __forceinline__ const unsigned short *cell_ptr(int ix, int iy, int iz) const
    {
        // ix in [-1, n-1]: brick of max(ix, 0), local index ix - E b + 1 in [0, E]
        const int bx = max(ix, 0) >> kShift, by = max(iy, 0) >> kShift, bz = max(iz, 0) >> kShift;
        const int lx = ix - (bx << kShift) + 1, ly = iy - (by << kShift) + 1, lz = iz - (bz << kShift) + 1;
        const Idx brick = ((Idx)bz * nby + by) * nbx + bx;
        return v + (brick * (Idx)kElems + (lz * S + ly) * S + lx);
    }

    template <bool CLAMP = true>
    __device__ __forceinline__ float nearest(long long X, long long Y, long long Z) const
    {
        int x = fx_round(X), y = fx_round(Y), z = fx_round(Z);
        if (CLAMP) {
            x = clampi(x, 0, nx - 1);
            y = clampi(y, 0, ny - 1);
            z = clampi(z, 0, nz - 1);
        } else {
            check_voxel(x, y, z, nx, ny, nz);
        }
        const int bx = x >> kShift, by = y >> kShift, bz = z >> kShift;
        const Idx brick = ((Idx)bz * nby + by) * nbx + bx;
        const unsigned short *p =
            v + (brick * (Idx)kElems + (((z & (E - 1)) + 1) * S + ((y & (E - 1)) + 1)) * S + (x & (E - 1)) + 1);
        return to_f32<T>(__ldg(p));
    }

    template <bool CLAMP = true>
    __device__ __forceinline__ void corners(int ix, int iy, int iz, float c[8]) const
    {
        check_range(ix, -1, nx - 1);
        check_range(iy, -1, ny - 1);
        check_range(iz, -1, nz - 1);
        const unsigned short *p = cell_ptr(ix, iy, iz);
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
        float c[8];
        corners<true>(cell_of<true>(X, nx), cell_of<true>(Y, ny), cell_of<true>(Z, nz), c);
        return trilerp(c, fx_frac(X), fx_frac(Y), fx_frac(Z));
    }
};

// Linear 16-bit cube [nz][ny][nx] (bfloat16 or binary16 raw values; fewer than 2^31
// voxels): the layout the staged marcher copies boxes from.  Values widen to FP32 on load.
template <typename T>
struct SamplerLin16 {
    static constexpr bool kLinearF32 = false;
    static constexpr bool kPair = false;
    const unsigned short *__restrict__ v;
    int nx, ny, nz;
    int sy, sz;  // strides of y and z in elements

    template <bool CLAMP = true>
    __device__ __forceinline__ float nearest(long long X, long long Y, long long Z) const
    {
        int x = fx_round(X), y = fx_round(Y), z = fx_round(Z);
        if (CLAMP) {
            x = clampi(x, 0, nx - 1);
            y = clampi(y, 0, ny - 1);
            z = clampi(z, 0, nz - 1);
        } else {
            check_voxel(x, y, z, nx, ny, nz);
        }
        return to_f32<T>(__ldg(v + (z * sz + y * sy + x)));
    }

    // corners of the cell with base (ix, iy, iz); CLAMP: each index in [-1, n-1]
    template <bool CLAMP = true>
    __device__ __forceinline__ void corners(int ix, int iy, int iz, float c[8]) const
    {
        if (!CLAMP) check_cell(ix, iy, iz, nx, ny, nz);
        int x0 = ix, y0 = iy, z0 = iz, dx = 1, dy = sy, dz = sz;
        if (CLAMP) {
            x0 = max(ix, 0);
            y0 = max(iy, 0);
            z0 = max(iz, 0);
            dx = min(ix + 1, nx - 1) - x0;
            dy = (min(iy + 1, ny - 1) - y0) * sy;
            dz = (min(iz + 1, nz - 1) - z0) * sz;
        }
        const unsigned short *p00 = v + (z0 * sz + y0 * sy + x0);
        const unsigned short *p01 = p00 + dy, *p10 = p00 + dz, *p11 = p10 + dy;
        c[0] = to_f32<T>(__ldg(p00));
        c[1] = to_f32<T>(__ldg(p00 + dx));
        c[2] = to_f32<T>(__ldg(p01));
        c[3] = to_f32<T>(__ldg(p01 + dx));
        c[4] = to_f32<T>(__ldg(p10));
        c[5] = to_f32<T>(__ldg(p10 + dx));
        c[6] = to_f32<T>(__ldg(p11));
        c[7] = to_f32<T>(__ldg(p11 + dx));
    }

    __device__ __forceinline__ float trilinear(long long X, long long Y, long long Z) const
    {
        float c[8];
        corners<true>(cell_of<true>(X, nx), cell_of<true>(Y, ny), cell_of<true>(Z, nz), c);
        return trilerp(c, fx_frac(X), fx_frac(Y), fx_frac(Z));
    }
};

// The two cubes of a line ratio in one linear 16-bit pair buffer: 32-bit elements
// [nz][ny][nx], low half the first cube.
template <typename T>
struct SamplerLin16Pair {
    static constexpr bool kLinearF32 = false;
    static constexpr bool kPair = true;
    const unsigned *__restrict__ v;
    int nx, ny, nz;
    int sy, sz;

    template <bool CLAMP = true>
    __device__ __forceinline__ float2 nearest2(long long X, long long Y, long long Z) const;  // (not instanced)

    template <bool CLAMP = true>
    __device__ __forceinline__ void corners2(int ix, int iy, int iz, float2 c[8]) const;
};

// The two cubes of a line ratio interleaved, float2 [nz][ny][nx]: (first, second) per voxel.
// One 8-byte load fetches a corner of both cubes; the interpolation runs on the pairs with
// packed FP32x2 lerps in the single-cube order, so each cube's value is bit-identical to
// trilerp() of that cube alone.
__device__ __forceinline__ float2 trilerp_pair(const float2 c[8], float fx, float fy, float fz)
{
    const float2 a = lerp2(c[0], c[1], fx), b = lerp2(c[2], c[3], fx);  // z0: rows y0, y1
    const float2 d = lerp2(c[4], c[5], fx), e = lerp2(c[6], c[7], fx);  // z1: rows y0, y1
    return lerp2(lerp2(a, b, fy), lerp2(d, e, fy), fz);
}

template <typename Idx>
struct SamplerF32Pair {
    static constexpr bool kLinearF32 = false;
    static constexpr bool kPair = true;
    const float2 *__restrict__ v;
    int nx, ny, nz;
    Idx sy, sz;  // strides of y and z in pairs

    template <bool CLAMP = true>
    __device__ __forceinline__ float2 nearest2(long long X, long long Y, long long Z) const
    {
        int x = fx_round(X), y = fx_round(Y), z = fx_round(Z);
        if (CLAMP) {
            x = clampi(x, 0, nx - 1);
            y = clampi(y, 0, ny - 1);
            z = clampi(z, 0, nz - 1);
        } else {
            check_voxel(x, y, z, nx, ny, nz);
        }
        return __ldg(v + ((Idx)z * sz + (Idx)y * sy + x));
    }

    template <bool CLAMP = true>
    __device__ __forceinline__ void corners2(int ix, int iy, int iz, float2 c[8]) const
    {
        if (!CLAMP) check_cell(ix, iy, iz, nx, ny, nz);
        int x0 = ix, y0 = iy, z0 = iz, dx = 1;
        Idx dy = sy, dz = sz;
        if (CLAMP) {
            x0 = max(ix, 0);
            y0 = max(iy, 0);
            z0 = max(iz, 0);
            dx = min(ix + 1, nx - 1) - x0;
            dy = (Idx)(min(iy + 1, ny - 1) - y0) * sy;
            dz = (Idx)(min(iz + 1, nz - 1) - z0) * sz;
        }
        const float2 *p00 = v + ((Idx)z0 * sz + (Idx)y0 * sy + x0);
        const float2 *p01 = p00 + dy, *p10 = p00 + dz, *p11 = p10 + dy;
        c[0] = __ldg(p00);
        c[1] = __ldg(p00 + dx);
        c[2] = __ldg(p01);
        c[3] = __ldg(p01 + dx);
        c[4] = __ldg(p10);
        c[5] = __ldg(p10 + dx);
        c[6] = __ldg(p11);
        c[7] = __ldg(p11 + dx);
    }
};

// One 32-bit element of the pair bricks -> (first, second) in FP32.
template <typename T>
__device__ __forceinline__ float2 pair_to_f32(unsigned w);
template <>
__device__ __forceinline__ float2 pair_to_f32<__nv_bfloat16>(unsigned w)
{
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <>
__device__ __forceinline__ float2 pair_to_f32<__half>(unsigned w)
{
    return __half22float2(__halves2half2(__ushort_as_half((unsigned short)(w & 0xffffu)),
                                         __ushort_as_half((unsigned short)(w >> 16))));
}

template <typename T>
template <bool CLAMP>
__device__ __forceinline__ float2 SamplerLin16Pair<T>::nearest2(long long X, long long Y, long long Z) const
{
    int x = fx_round(X), y = fx_round(Y), z = fx_round(Z);
    if (CLAMP) {
        x = clampi(x, 0, nx - 1);
        y = clampi(y, 0, ny - 1);
        z = clampi(z, 0, nz - 1);
    } else {
        check_voxel(x, y, z, nx, ny, nz);
    }
    return pair_to_f32<T>(__ldg(v + (z * sz + y * sy + x)));
}

template <typename T>
template <bool CLAMP>
__device__ __forceinline__ void SamplerLin16Pair<T>::corners2(int ix, int iy, int iz, float2 c[8]) const
{
    if (!CLAMP) check_cell(ix, iy, iz, nx, ny, nz);
    int x0 = ix, y0 = iy, z0 = iz, dx = 1, dy = sy, dz = sz;
    if (CLAMP) {
        x0 = max(ix, 0);
        y0 = max(iy, 0);
        z0 = max(iz, 0);
        dx = min(ix + 1, nx - 1) - x0;
        dy = (min(iy + 1, ny - 1) - y0) * sy;
        dz = (min(iz + 1, nz - 1) - z0) * sz;
    }
    const unsigned *p00 = v + (z0 * sz + y0 * sy + x0);
    const unsigned *p01 = p00 + dy, *p10 = p00 + dz, *p11 = p10 + dy;
    c[0] = pair_to_f32<T>(__ldg(p00));
    c[1] = pair_to_f32<T>(__ldg(p00 + dx));
    c[2] = pair_to_f32<T>(__ldg(p01));
    c[3] = pair_to_f32<T>(__ldg(p01 + dx));
    c[4] = pair_to_f32<T>(__ldg(p10));
    c[5] = pair_to_f32<T>(__ldg(p10 + dx));
    c[6] = pair_to_f32<T>(__ldg(p11));
    c[7] = pair_to_f32<T>(__ldg(p11 + dx));
}

// The pair storage as 32^3 bricks with the 1-voxel apron (layout of SamplerBrick), each
// element both cubes' 16-bit values.
template <typename T, typename Idx = long long>
struct SamplerBrickPair {
    static constexpr bool kLinearF32 = false;
    static constexpr bool kPair = true;
    const unsigned *__restrict__ v;
    int nx, ny, nz;
    int nbx, nby;

    static constexpr int S = kBrickStored;

    template <bool CLAMP = true>
    __device__ __forceinline__ float2 nearest2(long long X, long long Y, long long Z) const
    {
        int x = fx_round(X), y = fx_round(Y), z = fx_round(Z);
        if (CLAMP) {
            x = clampi(x, 0, nx - 1);
            y = clampi(y, 0, ny - 1);
            z = clampi(z, 0, nz - 1);
        } else {
            check_voxel(x, y, z, nx, ny, nz);
        }
        const int bx = x >> 5, by = y >> 5, bz = z >> 5;
        const Idx brick = ((Idx)bz * nby + by) * nbx + bx;
        const unsigned *p = v + (brick * (Idx)kBrickElems + (((z & 31) + 1) * S + ((y & 31) + 1)) * S + (x & 31) + 1);
        return pair_to_f32<T>(__ldg(p));
    }

    template <bool CLAMP = true>
    __device__ __forceinline__ void corners2(int ix, int iy, int iz, float2 c[8]) const
    {
        check_range(ix, -1, nx - 1);
        check_range(iy, -1, ny - 1);
        check_range(iz, -1, nz - 1);
        // ix in [-1, n-1]: brick of max(ix, 0), local index ix - 32 b + 1 in [0, 32]
        const int bx = max(ix, 0) >> 5, by = max(iy, 0) >> 5, bz = max(iz, 0) >> 5;
        const int lx = ix - (bx << 5) + 1, ly = iy - (by << 5) + 1, lz = iz - (bz << 5) + 1;
        const Idx brick = ((Idx)bz * nby + by) * nbx + bx;
        const unsigned *p = v + (brick * (Idx)kBrickElems + (lz * S + ly) * S + lx);
        c[0] = pair_to_f32<T>(__ldg(p));
        c[1] = pair_to_f32<T>(__ldg(p + 1));
        c[2] = pair_to_f32<T>(__ldg(p + S));
        c[3] = pair_to_f32<T>(__ldg(p + S + 1));
        c[4] = pair_to_f32<T>(__ldg(p + S * S));
        c[5] = pair_to_f32<T>(__ldg(p + S * S + 1));
        c[6] = pair_to_f32<T>(__ldg(p + S * S + S));
        c[7] = pair_to_f32<T>(__ldg(p + S * S + S + 1));
    }
};

// The pair sampler's corner cache (see CellCache below).
struct CellCachePair {
    int ix = -4, iy = -4, iz = -4;
    float2 c[8];
};

// 1: reuse the 8 corners of the cell a ray is in until it leaves that cell; 0: no reuse
#ifndef SHW_CELL_CACHE
#define SHW_CELL_CACHE 1
#endif

// The corners of the last interpolation cell a ray visited.  Consecutive samples
// 1/2 voxel apart often stay in one cell and then need no loads at all.
struct CellCache {
    int ix = -4, iy = -4, iz = -4;  // no cell yet: valid cells start at -1
    float c[8];
};

template <bool CLAMP, class S>
__device__ __forceinline__ float2 trilinear_pair_cached(const S &s, long long X, long long Y, long long Z,
                                                        CellCachePair &cc)
{
    const int ix = cell_of<CLAMP>(X, s.nx), iy = cell_of<CLAMP>(Y, s.ny), iz = cell_of<CLAMP>(Z, s.nz);
    if (!SHW_CELL_CACHE || ix != cc.ix || iy != cc.iy || iz != cc.iz) {
        s.template corners2<CLAMP>(ix, iy, iz, cc.c);
        cc.ix = ix;
        cc.iy = iy;
        cc.iz = iz;
    }
    return trilerp_pair(cc.c, fx_frac(X), fx_frac(Y), fx_frac(Z));
}

template <bool CLAMP, class S>
__device__ __forceinline__ float trilinear_cached(const S &s, long long X, long long Y, long long Z, CellCache &cc)
{
    const int ix = cell_of<CLAMP>(X, s.nx), iy = cell_of<CLAMP>(Y, s.ny), iz = cell_of<CLAMP>(Z, s.nz);
    if (!SHW_CELL_CACHE || ix != cc.ix || iy != cc.iy || iz != cc.iz) {
        s.template corners<CLAMP>(ix, iy, iz, cc.c);
        cc.ix = ix;
        cc.iy = iy;
        cc.iz = iz;
    }
    return trilerp(cc.c, fx_frac(X), fx_frac(Y), fx_frac(Z));
}

}  // namespace shw
