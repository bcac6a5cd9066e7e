// ray.cuh -- per-ray set-up: pixel -> ray (Appendix A), box clip, sample count
// (Algorithm 1's N and step), and the fixed-point sample positions used by the
// marchers.
//
// Precision design.  A ray of a 1024-deep cube spans ~2000 voxels; one float32
// ulp there is 1.2e-4 voxel, which after interpolation of unit-variance data
// would exceed the 1e-5-of-range accuracy target.  So the set-up is done once
// per ray in float-float arithmetic (an unevaluated sum hi + lo of two floats,
// ~48 significant bits; Dekker 1971 / Knuth TwoSum, products through FMA), and
// the sample positions are kept as 32.32 fixed-point integers: the start point
// P and the step D = h*d are rounded once to 2^-32 voxel, and sample k sits at
// P + k*D, an exact integer sum.  The integer part is the cell index, the top
// 23 fraction bits give the interpolation weight exactly.  No FP64 is used.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "shw.h"

namespace shw {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff1(float a) { return {a, 0.0f}; }

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ ff two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Dekker's FastTwoSum, valid for |a| >= |b|.
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// p + e == a * b exactly (the FMA computes the rounding error of the product).
__device__ __forceinline__ ff two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// Long division with two correction steps.
__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff r = ff_sub(a, ff_mul(ff1(q1), b));
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = ff_sub(r, ff_mul(ff1(q2), b));
    float q3 = __fdiv_rn(r.hi, b.hi);
    return ff_add(fast_two_sum(q1, q2), ff1(q3));
}

// One Newton step on the float square root.
__device__ __forceinline__ ff ff_sqrt(ff a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    float x = __fsqrt_rn(a.hi);
    ff r = ff_sub(a, two_prod(x, x));
    float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, x));
    return fast_two_sum(x, c);
}

__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_lt(b, a) ? b : a; }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }

// floor of a float-float as an integer (|x| < 2^30).
__device__ __forceinline__ int ff_floor_int(ff x)
{
    float f = floorf(x.hi);
    int i = __float2int_rz(f);
    if (f == x.hi) {  // hi is an integer: the sign of lo decides
        float g = floorf(x.lo);
        i += __float2int_rz(g);
    }
    return i;
}

// Round a float-float to the nearest multiple of 2^-32, as an integer count.
__device__ __forceinline__ long long ff_to_fx(ff v)
{
    return __float2ll_rn(__fmul_rn(v.hi, 4294967296.0f)) + __float2ll_rn(__fmul_rn(v.lo, 4294967296.0f));
}

// A ray in 32.32 fixed point: sample k is at P + k*D; N samples; U: the unit
// direction (one voxel along the ray).
struct RayFx {
    long long P[3];
    long long D[3];
    long long U[3];
    int N;
};

// Pixel (px, py) of camera c -> origin o and unit direction d (Appendix A).
__device__ __forceinline__ void pixel_ray_ff(const shw_camera &c, int px, int py, ff o[3], ff d[3])
{
    const ff W = ff1((float)c.width), H = ff1((float)c.height);
    const ff xs = ff_div(ff1((float)(2 * px + 1 - c.width)), W);   // 2(px+1/2)/W - 1
    const ff ys = ff_div(ff1((float)(c.height - 2 * py - 1)), H);  // 1 - 2(py+1/2)/H
    const ff aspect = ff_div(W, H);
    if (c.ortho) {
        const ff hh = ff1(c.ortho_half_h);
        const ff hw = ff_mul(hh, aspect);
        const ff sx = ff_mul(xs, hw), sy = ff_mul(ys, hh);
        ff n2 = ff_add(ff_add(two_prod(c.fwd[0], c.fwd[0]), two_prod(c.fwd[1], c.fwd[1])),
                       two_prod(c.fwd[2], c.fwd[2]));
        const ff nf = ff_sqrt(n2);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = ff_add(ff_add(ff1(c.eye[a]), ff_mul(sx, ff1(c.right[a]))), ff_mul(sy, ff1(c.up[a])));
            d[a] = ff_div(ff1(c.fwd[a]), nf);
        }
    } else {
        const ff th = ff1(c.tan_half_fovy);
        const ff tx = ff_mul(ff_mul(xs, th), aspect), ty = ff_mul(ys, th);
        ff u[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            u[a] = ff_add(ff_add(ff1(c.fwd[a]), ff_mul(tx, ff1(c.right[a]))), ff_mul(ty, ff1(c.up[a])));
        const ff nu = ff_sqrt(ff_add(ff_add(ff_mul(u[0], u[0]), ff_mul(u[1], u[1])), ff_mul(u[2], u[2])));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = ff1(c.eye[a]);
            d[a] = ff_div(u[a], nu);
        }
    }
}

// Clip to the closed box [-0.5, n-0.5]^3 and t >= 0, count N = floor((t1-t0)/h)
// samples, and express sample positions in fixed point.  Returns false on a miss.
__device__ __forceinline__ bool setup_ray(const shw_camera &c, int px, int py, int nx, int ny, int nz,
                                          float h, RayFx &r)
{
    ff o[3], d[3];
    pixel_ray_ff(c, px, py, o, d);
    const int n[3] = {nx, ny, nz};
    ff tmin = ff1(0.0f), tmax = ff1(0.0f);
    bool has_min = false, has_max = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const ff lo = ff1(-0.5f), hi = ff1((float)n[a] - 0.5f);
        if (d[a].hi == 0.0f) {
            if (ff_lt(o[a], lo) || ff_lt(hi, o[a])) {
                r.N = 0;
                return false;
            }
            continue;
        }
        ff ta = ff_div(ff_sub(lo, o[a]), d[a]);
        ff tb = ff_div(ff_sub(hi, o[a]), d[a]);
        ff tn = ff_min(ta, tb), tf = ff_max(ta, tb);
        tmin = has_min ? ff_max(tmin, tn) : tn;
        tmax = has_max ? ff_min(tmax, tf) : tf;
        has_min = has_max = true;
    }
    const ff t0 = (has_min && ff_lt(ff1(0.0f), tmin)) ? tmin : ff1(0.0f);  // keep t >= 0
    if (!has_max || !ff_lt(t0, tmax)) {
        r.N = 0;
        return false;
    }
    const ff hf = ff1(h);
    const int N = ff_floor_int(ff_div(ff_sub(tmax, t0), hf));
    r.N = N > 0 ? N : 0;
    if (r.N == 0) return false;
    const ff ts = ff_add(t0, ff1(0.5f * h));  // first sample at t0 + h/2 (h/2 exact)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.P[a] = ff_to_fx(ff_add(o[a], ff_mul(ts, d[a])));
        r.D[a] = ff_to_fx(ff_mul(hf, d[a]));
        r.U[a] = ff_to_fx(d[a]);
    }
    return true;
}

// Cell index and interpolation weight of one fixed-point coordinate.
__device__ __forceinline__ int fx_cell(long long p) { return (int)(p >> 32); }
__device__ __forceinline__ float fx_frac(long long p)
{
    // the 23 most significant fraction bits as the mantissa of a float in [1, 2): lo >> 9 is
    // below 2^23, so OR-ing the exponent in equals adding it
    return __uint_as_float(((unsigned)p >> 9) | 0x3f800000u) - 1.0f;
}
// The next sample's position: X + D, exactly.  (A plain 64-bit addition: a form built from
// inline multiply-adds, meant to move the work to the FMA pipe, cost register moves around
// every use.)
__device__ __forceinline__ long long fx_step(long long X, long long D) { return X + D; }

// floor(p + 1/2): the nearest voxel (round half up).
__device__ __forceinline__ int fx_round(long long p) { return (int)((p + 0x80000000LL) >> 32); }

}  // namespace shw
