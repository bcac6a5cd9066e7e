// render_impl.cuh -- the ray marcher: one thread per pixel (= one ray, the
// fragment of Section 2.3), Algorithm 1's loop with one transfer function.
//
// Thread layout: a CTA of 64 threads (two warps) renders a small pixel tile, so the
// hardware's CTA scheduler balances rays of very different lengths finely.  A warp
// covers a 16 x 2, 2 x 16 or 8 x 4 pixel tile, elongated along the image axis that
// runs closest to the cube's contiguous x axis so its loads share cache lines.
//
// Per ray: an FP32 test rejects rays that clearly miss the box; the exact set-up
// (float-float, ray.cuh) gives N and the fixed-point start and step; the samples
// are split into a clamped head, a clamp-free interior (cells in [0, n-2] on
// every axis, verified exactly in integer arithmetic) and a clamped tail.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "ray.cuh"
#include "sampler.cuh"

namespace shw {

struct RenderArgs {
    float4 *rgba;       // [H][W]
    float *scalar;      // [H][W] or null
    int *index;         // [H][W] or null
    int *nsamples;      // [H][W] or null
    float *ckpt_T;      // COMPOSITE checkpoints: [nckpt][H][W] or null
    int *ckpt_K;        // [H][W] samples processed, or null
    const float4 *lut;  // [256]
    int width, height;
    int nckpt, ckpt_interval;
    int nmax;        // upper bound of N over all rays (box diagonal / step + 1)
    int warp_shift;  // log2 of the warp tile's width
    int tiles_x, tiles_y;  // CTA tiles per image row / column
    int ctx, cty;          // the tile holding the projected cube centre (dispatched first)
    float step, lo, inv_range, opacity_scale, term_alpha, ratio_floor;
    int nx, ny, nz;
    int filter, alpha_thr;  // shw_filter; the alpha-threshold option of spectral / first-moment colouring
    float tmin, tmax, tinv; // the filter's thresholds; 1 / (tmax - tmin) for domain scaling
    int smooth;             // shw_smooth_kind of in-ray smoothing
    int box_lattice;        // 2: box smoothing with a step of exactly 1/2 voxel runs as running sums
    int smooth_n;           // box: neighbours on each side; taps: fetches on each side per axis
    float smooth_c0;        // box: 1 / (2 arm + 1); taps: weight of the value entering each axis pass
    float smooth_w[SHW_MAX_SMOOTH_TAPS];          // taps: weights
    long long smooth_off[SHW_MAX_SMOOTH_TAPS];    // taps: offsets, 32.32 fixed point
};


#ifndef SHW_CTA_WARPS
#define SHW_CTA_WARPS 2
#endif
#ifndef SHW_LUT_SMEM
#define SHW_LUT_SMEM 0  // 1: compositing stages the colour map in shared memory; 0: reads it through L1
#endif
constexpr int kCtaWarps = SHW_CTA_WARPS, kRenderThreads = 32 * SHW_CTA_WARPS;
#ifndef SHW_WARP_SHIFT
#define SHW_WARP_SHIFT -1  // -1: chosen per launch from the camera; else log2 of the warp tile width
#endif

// Colour-map lookup: linear between the 256 knots at u = 255 v_hat (Section 2.1).
__device__ __forceinline__ float4 lut_eval(const float4 *L, float vhat)
{
    const float u = vhat * 255.0f;
    const int i0 = min(__float2int_rd(u), 254);
    const float f = u - (float)i0;
    const float4 a = L[i0], b = L[i0 + 1];
    // four lerps as two packed FP32x2 ones (the same rounding as scalar lerps)
    const float2 rg = lerp2(make_float2(a.x, a.y), make_float2(b.x, b.y), f);
    const float2 ba = lerp2(make_float2(a.z, a.w), make_float2(b.z, b.w), f);
    return make_float4(rg.x, rg.y, ba.x, ba.y);
}

__device__ __forceinline__ float normalise(float v, float lo, float inv_range)
{
    // clamped to [0, 1] by one saturating operation; a NaN argument yields 0 (never reached:
    // NaN samples become lo)
    return __saturatef((v - lo) * inv_range);
}

// The per-sample filter of Algorithm 1: Algorithm 10 (intensity clipping) replaces a value
// below tmin or above tmax by DATAMIN; Algorithm 11 (domain scaling) does the same and
// maps [tmin, tmax] onto [0, 1].  A NaN passes through (and becomes DATAMIN later).
__device__ __forceinline__ float filter_value(float v, const RenderArgs &a)
{
    if (a.filter == SHW_FILTER_NONE) return v;
    const bool out = v < a.tmin || v > a.tmax;
    if (a.filter == SHW_FILTER_CLIP) return out ? a.lo : v;
    return out ? a.lo : __fmul_rn(__fsub_rn(v, a.tmin), a.tinv);
}

// Alpha of the first-moment-inspired colourings: the value's place in the colour-map
// domain, or with the threshold option transparent up to tmin and opaque above.
__device__ __forceinline__ float colour_alpha(float v, const RenderArgs &a)
{
    return a.alpha_thr ? (v > a.tmin ? 1.0f : 0.0f) : normalise(v, a.lo, a.inv_range);
}

// CTA tile: the CTA's warps stacked across the warp tile's short side.
__host__ __device__ __forceinline__ void cta_tile(int ws, int &tw, int &th)
{
    const int wtx = 1 << ws, wty = 32 >> ws;
    tw = wtx >= wty ? wtx : kCtaWarps * wtx;
    th = wtx >= wty ? kCtaWarps * wty : wty;
}

// k-th element of c, c-1, c+1, c-2, c+2, ... restricted to [0, n): a centre-out order
__host__ __device__ __forceinline__ int centre_out(int k, int c, int n)
{
    const int m = c < n - 1 - c ? c : n - 1 - c;  // rings that fit on both sides
    if (k <= 2 * m) return (k & 1) ? c - (k + 1) / 2 : c + k / 2;
    const int rest = k - 2 * m;  // then the longer side, moving outwards
    return c - m > 0 ? c - m - rest : c + m + rest;
}

// Tiles are dispatched centre-out (rows, then columns within a row, from the tile
// under the projected cube centre), so the longest rays start first and short or
// empty tiles fill the end of the launch.
__device__ __forceinline__ void tile_pixel(int &px, int &py, const RenderArgs &a)
{
    const int ws = a.warp_shift, wtx = 1 << ws, wty = 32 >> ws;
    int tw, th;
    cta_tile(ws, tw, th);
    const int rank = blockIdx.x, rr = rank / a.tiles_x, cr = rank - rr * a.tiles_x;
    const int ty = centre_out(rr, a.cty, a.tiles_y), tx = centre_out(cr, a.ctx, a.tiles_x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    px = tx * tw + (wtx >= wty ? 0 : warp * wtx) + (lane & (wtx - 1));
    py = ty * th + (wtx >= wty ? warp * wty : 0) + (lane >> ws);
}

// Conservative FP32 rejection: true only if the ray surely misses the box (the box
// is widened by a margin far larger than the FP32 error of the ray).
__device__ __forceinline__ bool quick_miss(const shw_camera &c, int px, int py, int nx, int ny, int nz)
{
    const float W = (float)c.width, H = (float)c.height;
    const float xs = (float)(2 * px + 1 - c.width) / W, ys = (float)(c.height - 2 * py - 1) / H;
    const float aspect = W / H;
    float o[3], d[3];
    if (c.ortho) {
        const float sx = xs * c.ortho_half_h * aspect, sy = ys * c.ortho_half_h;
        for (int k = 0; k < 3; ++k) {
            o[k] = c.eye[k] + sx * c.right[k] + sy * c.up[k];
            d[k] = c.fwd[k];
        }
    } else {
        const float tx = xs * c.tan_half_fovy * aspect, ty = ys * c.tan_half_fovy;
        for (int k = 0; k < 3; ++k) {
            o[k] = c.eye[k];
            d[k] = c.fwd[k] + tx * c.right[k] + ty * c.up[k];
        }
    }
    const int n[3] = {nx, ny, nz};
    float tmin = -INFINITY, tmax = INFINITY;
    for (int k = 0; k < 3; ++k) {
        const float m = 0.05f + 1e-5f * fabsf(o[k]);
        const float lo = -0.5f - m, hi = (float)n[k] - 0.5f + m;
        if (d[k] == 0.0f) {
            if (o[k] < lo || o[k] > hi) return true;
            continue;
        }
        const float t1 = (lo - o[k]) / d[k], t2 = (hi - o[k]) / d[k];
        tmin = fmaxf(tmin, fminf(t1, t2));
        tmax = fminf(tmax, fmaxf(t1, t2));
    }
    return tmax < tmin || tmax < 0.0f;
}

// Samples k in [ka, kb) whose cells lie in [0, n-2] on every axis.  An FP32
// estimate, then exact integer checks of both ends (cells move monotonically along
// a ray, so valid ends make the whole range valid).  Empty range: ka = kb = N.
__device__ __forceinline__ void interior_range(const RayFx &r, int nx, int ny, int nz, int N, int &ka, int &kb)
{
    const int n[3] = {nx, ny, nz};
    ka = 0;
    kb = N;
    for (int a = 0; a < 3; ++a) {
        const long long P = r.P[a], D = r.D[a], U = (long long)(n[a] - 1) << 32;
        if (D == 0) {
            if (!(P >= 0 && P < U)) {
                ka = kb = N;
                return;
            }
            continue;
        }
        const float p = __ll2float_rn(P) * 2.3283064365386963e-10f, d = __ll2float_rn(D) * 2.3283064365386963e-10f;
        const float u = (float)(n[a] - 1);
        const float t0 = (d > 0.0f ? -p : u - p) / d, t1 = (d > 0.0f ? u - p : -p) / d;
        ka = max(ka, (int)fminf(fmaxf(ceilf(t0), 0.0f), (float)N));
        kb = min(kb, (int)fminf(fmaxf(ceilf(t1), 0.0f), (float)N));
    }
    auto inside = [&](int k) {
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const long long q = r.P[a] + (long long)k * r.D[a];
            ok = ok && q >= 0 && q < ((long long)(n[a] - 1) << 32);
        }
        return ok;
    };
    for (int i = 0; i < 4 && ka < kb && !inside(ka); ++i) ++ka;
    for (int i = 0; i < 4 && kb > ka && !inside(kb - 1); ++i) --kb;
    if (ka >= kb || !inside(ka) || !inside(kb - 1)) ka = kb = N;
}

template <int INTERP, class S>
__device__ __forceinline__ float fetch(const S &s, long long X, long long Y, long long Z)
{
    if constexpr (INTERP == SHW_NEAREST)
        return s.template nearest<true>(X, Y, Z);
    else
        return s.trilinear(X, Y, Z);
}

template <bool CLAMP, int INTERP, class S>
__device__ __forceinline__ float sample(const S &s, long long X, long long Y, long long Z, CellCache &cc)
{
    if constexpr (INTERP == SHW_NEAREST)
        return s.template nearest<CLAMP>(X, Y, Z);
    else
        return trilinear_cached<CLAMP>(s, X, Y, Z, cc);
}

// Algorithm 1's "val <- smooth(val)" on one cube at (X, Y, Z) (Sections 4.1-4.2).
// Box (Algorithm 8): the sample and a.smooth_n neighbours on each side one voxel apart
// along the ray (U, the unit direction), times 1 / (2 arm + 1).  Taps (Algorithm 9 per
// data axis): passes along x, y, z in turn, each val <- c0 val + sum_j w_j (v(+off_j) +
// v(-off_j)).  The centre goes through the cell cache; taps fetch with clamping.
template <int INTERP, class S>
__device__ __forceinline__ float smoothed_sample(const S &s, long long X, long long Y, long long Z,
                                                 const long long U[3], const RenderArgs &a, CellCache &cc)
{
    float v = sample<true, INTERP>(s, X, Y, Z, cc);
    if (a.smooth == SHW_SMOOTH_BOX) {
        long long ox = 0, oy = 0, oz = 0;
        for (int i = 0; i < a.smooth_n; ++i) {
            ox += U[0];
            oy += U[1];
            oz += U[2];
            v += fetch<INTERP>(s, X + ox, Y + oy, Z + oz);
            v += fetch<INTERP>(s, X - ox, Y - oy, Z - oz);
        }
        v *= a.smooth_c0;
    } else if (a.smooth == SHW_SMOOTH_TAPS) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float out = v * a.smooth_c0;
            for (int j = 0; j < a.smooth_n; ++j) {
                const long long o = a.smooth_off[j];
                const long long dx = ax == 0 ? o : 0, dy = ax == 1 ? o : 0, dz = ax == 2 ? o : 0;
                out = __fmaf_rn(fetch<INTERP>(s, X + dx, Y + dy, Z + dz), a.smooth_w[j], out);
                out = __fmaf_rn(fetch<INTERP>(s, X - dx, Y - dy, Z - dz), a.smooth_w[j], out);
            }
            v = out;
        }
    }
    return v;
}

// One cube's value at a ray sample: smoothed (SM) or the plain fetch.
template <bool CLAMP, bool SM, int INTERP, class S>
__device__ __forceinline__ float ray_sample(const S &s, long long X, long long Y, long long Z, CellCache &cc,
                                            const RenderArgs &a, const long long *U)
{
    if constexpr (SM)
        return smoothed_sample<INTERP>(s, X, Y, Z, U, a, cc);
    else
        return sample<CLAMP, INTERP>(s, X, Y, Z, cc);
}

// Both cubes of a line ratio at one sample from the interleaved pair storage.
template <bool CLAMP, int INTERP, class S>
__device__ __forceinline__ float2 pair_sample(const S &s, long long X, long long Y, long long Z, CellCachePair &cc)
{
    if constexpr (INTERP == SHW_NEAREST)
        return s.template nearest2<CLAMP>(X, Y, Z);
    else
        return trilinear_pair_cached<CLAMP>(s, X, Y, Z, cc);
}

template <class S>
using CacheOf = typename std::conditional<S::kPair, CellCachePair, CellCache>::type;

// The two cubes' raw values at a sample of the line ratios: one interleaved fetch for the
// pair storage, else one fetch (or smoothed value) per cube.
template <bool CLAMP, bool SM, int INTERP, class S, class CC>
__device__ __forceinline__ void two_samples(const S &s, const S &s2, long long X, long long Y, long long Z, CC &cc,
                                            CC &cc2, const RenderArgs &a, const long long *U, float &c1, float &c2)
{
    if constexpr (S::kPair) {
        const float2 c = pair_sample<CLAMP, INTERP>(s, X, Y, Z, cc);
        c1 = c.x;
        c2 = c.y;
    } else {
        c1 = ray_sample<CLAMP, SM, INTERP>(s, X, Y, Z, cc, a, U);
        c2 = ray_sample<CLAMP, SM, INTERP>(s2, X, Y, Z, cc2, a, U);
    }
}

// ---- in-ray box smoothing on the ray's own sample lattice ---------------------

#ifndef SHW_BOX_RESUM
#define SHW_BOX_RESUM 64  // the running sums are recomputed directly every this many samples of a class
#endif

// Box smoothing (Algorithm 8) when the step is exactly 1/M voxel (M = 2 is instanced): the neighbours of sample
// k one voxel apart along the ray are the samples k +- i M of the same ray (P + j D, exact in
// fixed point; M D equals the unit direction to 2^-32 voxel).  The box value of sample k is a
// sum over the lattice class of k, kept as M running sums: sum(k) = sum(k - M) + r(k + arm M)
// - r(k - (arm + 1) M), two fetches per sample instead of 2 arm + 1.  A sum is recomputed
// directly every SHW_BOX_RESUM samples of its class (bounding rounding drift) and whenever it
// is not finite (a NaN or infinite tap inside the window gives the direct definition's value).
template <int M, int MODE, int INTERP, class S, class St>
__device__ __forceinline__ void march_box_lattice(const S &s, const RenderArgs &a, St &st, const long long P[3],
                                                  const long long D[3], int N, int &kdone)
{
    const int arm = a.smooth_n;
    CellCache ca, cb, cd;  // leading, trailing and direct fetches: each walks the ray monotonically
    auto raw = [&](int j, CellCache &cc) {
        return sample<true, INTERP>(s, P[0] + (long long)j * D[0], P[1] + (long long)j * D[1],
                                    P[2] + (long long)j * D[2], cc);
    };
    auto direct = [&](int k) {  // the definition's order: the sample, then the pairs +-i
        float t = raw(k, cd);
        for (int i = 1; i <= arm; ++i) {
            t += raw(k + i * M, cd);
            t += raw(k - i * M, cd);
        }
        return t;
    };
    float sum[M];
    for (int k0 = 0; k0 < N; k0 += M) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const int k = k0 + c;
            if (k >= N) break;
            float t;
            if (k0 == 0 || (k0 / M) % SHW_BOX_RESUM == 0) {
                t = direct(k);
            } else {
                t = sum[c] + raw(k + arm * M, ca) - raw(k - (arm + 1) * M, cb);
                if (!isfinite(t)) t = direct(k);
            }
            sum[c] = t;
            float v = t * a.smooth_c0;
            v = filter_value(isnan(v) ? a.lo : v, a);
            v = isnan(v) ? a.lo : v;  // a NaN sample counts as DATAMIN
            if (st.update(v, k)) {
                kdone = k + 1;
                return;
            }
        }
    }
    kdone = N;
}

// ---- transfer-function state per mode --------------------------------------

// Eq. 1 / Algorithms 2, 4, 14: running maximum with ">=" (the last maximum wins)
struct MaxState {
    float m = -INFINITY;
    int kmax = 0;
    __device__ __forceinline__ bool update(float v, int k)
    {
        if (v >= m) {
            m = v;
            kmax = k;
        }
        return false;
    }
};

// MIP when no channel (argmax) output is wanted: the running maximum alone.  A NaN sample
// has already been replaced by DATAMIN, so fmaxf sees numbers only and gives the same value
// as the ordered >= update (the two can differ only in the sign of a zero maximum).
constexpr int kMipValue = 16;
struct MaxValState {
    float m = -INFINITY;
    int kmax = 0;
    __device__ __forceinline__ bool update(float v, int)
    {
        m = fmaxf(m, v);
        return false;
    }
};

// Eq. 3 divided by N; compensated (Kahan) summation keeps FP32 accurate
struct AvgState {
    float sum = 0.0f, comp = 0.0f;
    __device__ __forceinline__ bool update(float v, int)
    {
        const float y = __fsub_rn(v, comp);
        const float t = __fadd_rn(sum, y);
        comp = __fsub_rn(__fsub_rn(t, sum), y);
        sum = t;
        return false;
    }
};

// Algorithm 3 in premultiplied form; stops after the sample that makes alpha > term
// A sample's position along one axis as colouring uses it: the voxel for nearest
// sampling, the point itself for trilinear (fixed point -> FP32); and its texture
// coordinate (p + 1/2) / n in [0, 1].
__device__ __forceinline__ float colour_pos(long long P, int n, bool nearest)
{
    return nearest ? (float)clampi(fx_round(P), 0, n - 1) : __fadd_rn((float)fx_cell(P), fx_frac(P));
}
__device__ __forceinline__ float tex_coord(float p, int n) { return __saturatef((p + 0.5f) / (float)n); }

constexpr int kColourValue = 0, kColourSpectral = 1, kColourPosition = 2;

// Algorithm 3 in premultiplied form; stops after the sample that makes alpha > term.
// The colour comes from the value (Algorithm 3), from the map at the sample's spectral
// position (Algorithm 5, AVIP_1) or from its position (Algorithm 7, AVIP_RGB); the
// position then advances with the samples, which arrive in order.
template <int COLOUR>
struct CompositeStateT {
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    const float4 *lut;
    float lo, inv_range, s, term;
    float *ckpt;  // this ray's first checkpoint slot, or null
    long long ckpt_stride;
    int I, nckpt;
    long long X = 0, Y = 0, Z = 0, DX = 0, DY = 0, DZ = 0;  // COLOUR != value: the sample's position
    int nx = 1, ny = 1, nz = 1;
    bool nearest = false;
    __device__ __forceinline__ bool update(float v, int k)
    {
        if (ckpt != nullptr && (k % I) == 0 && k / I < nckpt) ckpt[(long long)(k / I) * ckpt_stride] = T;
        const float4 c = lut_eval(lut, normalise(v, lo, inv_range));
        float r = c.x, g = c.y, b = c.z;
        if constexpr (COLOUR == kColourSpectral) {
            const float4 q = lut_eval(lut, tex_coord(colour_pos(Z, nz, nearest), nz));
            r = q.x;
            g = q.y;
            b = q.z;
        } else if constexpr (COLOUR == kColourPosition) {
            r = tex_coord(colour_pos(Z, nz, nearest), nz);
            g = tex_coord(colour_pos(Y, ny, nearest), ny);
            b = tex_coord(colour_pos(X, nx, nearest), nx);
        }
        if constexpr (COLOUR != kColourValue) {
            X += DX;
            Y += DY;
            Z += DZ;
        }
        const float al = __saturatef(s * c.w);
        const float w = T * al;
        cr = __fmaf_rn(w, r, cr);
        cg = __fmaf_rn(w, g, cg);
        cb = __fmaf_rn(w, b, cb);
        T = T * (1.0f - al);
        return 1.0f - T > term;
    }
};
using CompositeState = CompositeStateT<kColourValue>;

// Algorithms 12-13 (line ratio, Method 1): each cube's running maximum (">")
struct RatioMaxState {
    float m1 = -INFINITY, m2 = -INFINITY;
    int kmax = 0;
    __device__ __forceinline__ void update2(float c1, float c2)
    {
        if (c1 > m1) m1 = c1;
        if (c2 > m2) m2 = c2;
    }
};

template <int MODE>
constexpr bool is_composite = MODE == SHW_COMPOSITE || MODE == SHW_COMPOSITE_SPECTRAL || MODE == SHW_COMPOSITE_RGB;
template <int MODE>
constexpr bool two_cubes = MODE == SHW_RATIO || MODE == SHW_RATIO_MIP;

// Eq. 4 along the ray: intensity-weighted mean height.  Weights are the intensity above
// DATAMIN (NaN samples are DATAMIN already); the height is the sample's z (its channel
// for nearest sampling).  Compensated sums of w, z w and v (for the mean that sets alpha).
// Z advances with the samples, which arrive in order.
struct MomentState {
    float sw = 0.0f, cw = 0.0f, szw = 0.0f, cz = 0.0f, sv = 0.0f, cv = 0.0f;
    long long Z = 0, DZ = 0;
    float lo = 0.0f;
    int nz = 1;
    bool nearest = false;
    __device__ __forceinline__ static void kahan(float &s, float &c, float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ bool update(float v, int)
    {
        const float z = nearest ? (float)clampi(fx_round(Z), 0, nz - 1) : __fadd_rn((float)fx_cell(Z), fx_frac(Z));
        const float w = fmaxf(__fsub_rn(v, lo), 0.0f);
        kahan(sw, cw, w);
        kahan(szw, cz, __fmul_rn(z, w));
        kahan(sv, cv, v);
        Z += DZ;
        return false;
    }
};

template <int MODE>
struct StateOf {
    using type = MaxState;
};
template <>
struct StateOf<SHW_MOMENT1> {
    using type = MomentState;
};
template <>
struct StateOf<kMipValue> {
    using type = MaxValState;
};
template <>
struct StateOf<SHW_AVG> {
    using type = AvgState;
};
template <>
struct StateOf<SHW_COMPOSITE> {
    using type = CompositeState;
};
template <>
struct StateOf<SHW_COMPOSITE_SPECTRAL> {
    using type = CompositeStateT<kColourSpectral>;
};
template <>
struct StateOf<SHW_COMPOSITE_RGB> {
    using type = CompositeStateT<kColourPosition>;
};
template <>
struct StateOf<SHW_RATIO_MIP> {
    using type = RatioMaxState;
};

// Samples [k0, k1) of one ray; true if the transfer function stopped the ray
// (then kdone = samples processed).  X, Y, Z advance with the samples.
// SM: every sample smoothed (U: the ray's unit direction).
template <bool CLAMP, int MODE, int INTERP, bool SM = false, class S, class St, class CC>
__device__ __forceinline__ bool march(const S &s, const S &s2, const RenderArgs &a, St &st, CC &cc,
                                      CC &cc2, long long &X, long long &Y, long long &Z, long long DX,
                                      long long DY, long long DZ, int k0, int k1, int &kdone,
                                      const long long *U = nullptr)
{
    for (int k = k0; k < k1; ++k) {
        if constexpr (MODE == SHW_RATIO_MIP) {
            // Algorithm 13: each cube's maximum; a NaN sample counts as DATAMIN
            float r1, r2;
            two_samples<CLAMP, SM, INTERP>(s, s2, X, Y, Z, cc, cc2, a, U, r1, r2);
            const float c1 = filter_value(r1, a), c2 = filter_value(r2, a);
            st.update2(isnan(c1) ? a.lo : c1, isnan(c2) ? a.lo : c2);
        } else {
            float v;
            if constexpr (MODE == SHW_RATIO) {
                // Algorithm 14: ratio where cube1 exceeds the floor, else DATAMIN
                float r1, r2;
                two_samples<CLAMP, SM, INTERP>(s, s2, X, Y, Z, cc, cc2, a, U, r1, r2);
                const float c1 = filter_value(r1, a), c2 = filter_value(r2, a);
                v = (c1 > a.ratio_floor) ? __fdiv_rn(c2, c1) : a.lo;
            } else {
                v = ray_sample<CLAMP, SM, INTERP>(s, X, Y, Z, cc, a, U);
                v = filter_value(isnan(v) ? a.lo : v, a);
            }
            v = isnan(v) ? a.lo : v;  // a NaN sample counts as DATAMIN
            if (st.update(v, k)) {
                kdone = k + 1;
                return true;
            }
        }
        X += DX;
        Y += DY;
        Z += DZ;
    }
    kdone = k1;
    return false;
}

#ifndef SHW_PREFETCH
#define SHW_PREFETCH 1  // 1: the interior loop loads the next cell's corners a sample ahead
#endif

// The interior samples [k0, k1) (every cell in [0, n-2] on every axis, no clamping),
// trilinear, software-pipelined: while sample k is interpolated and fed to the
// transfer function, the corners of sample k+1's cell are already being loaded when
// that cell differs.  Same arithmetic as march<false>, so the same results.
// march_interior_pair: the line ratios on the interleaved pair storage, one 8-byte load per
// corner for both cubes, packed interpolation (each cube bit-identical to the single form).
template <int MODE, class S, class St>
__device__ __forceinline__ bool march_interior_pair(const S &s, const RenderArgs &a, St &st, long long &X,
                                                    long long &Y, long long &Z, long long DX, long long DY,
                                                    long long DZ, int k0, int k1, int &kdone)
{
    if (k0 >= k1) {
        kdone = k1;
        return false;
    }
    int cx = fx_cell(X), cy = fx_cell(Y), cz = fx_cell(Z);
    float2 cur[8];
    s.template corners2<false>(cx, cy, cz, cur);
    for (int k = k0; k < k1; ++k) {
        const long long Xn = X + DX, Yn = Y + DY, Zn = Z + DZ;
        const int nx = fx_cell(Xn), ny = fx_cell(Yn), nz = fx_cell(Zn);
        const bool pf = ((nx != cx) | (ny != cy) | (nz != cz)) && k + 1 < k1;
        float2 nxt[8];
        if (pf) s.template corners2<false>(nx, ny, nz, nxt);
        const float2 c = trilerp_pair(cur, fx_frac(X), fx_frac(Y), fx_frac(Z));
        const float c1 = filter_value(c.x, a), c2 = filter_value(c.y, a);
        if constexpr (MODE == SHW_RATIO_MIP) {
            st.update2(isnan(c1) ? a.lo : c1, isnan(c2) ? a.lo : c2);
        } else {
            // Algorithm 14: ratio where cube1 exceeds the floor, else DATAMIN
            float v = (c1 > a.ratio_floor) ? __fdiv_rn(c2, c1) : a.lo;
            v = isnan(v) ? a.lo : v;
            if (st.update(v, k)) {
                kdone = k + 1;
                return true;
            }
        }
        if (pf) {
#pragma unroll
            for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
            cx = nx;
            cy = ny;
            cz = nz;
        }
        X = Xn;
        Y = Yn;
        Z = Zn;
    }
    kdone = k1;
    return false;
}

// march_interior_single: one or two separate cubes.
template <int MODE, class S, class St>
__device__ __forceinline__ bool march_interior_single(const S &s, const S &s2, const RenderArgs &a, St &st,
                                                      long long &X, long long &Y, long long &Z, long long DX,
                                                      long long DY, long long DZ, int k0, int k1, int &kdone)
{
    constexpr bool TWO = two_cubes<MODE>;
    if (k0 >= k1) {
        kdone = k1;
        return false;
    }
    int cx = fx_cell(X), cy = fx_cell(Y), cz = fx_cell(Z);
    float cur[8], cur2[8];
    s.template corners<false>(cx, cy, cz, cur);
    if constexpr (TWO) s2.template corners<false>(cx, cy, cz, cur2);
    for (int k = k0; k < k1; ++k) {
        const long long Xn = X + DX, Yn = Y + DY, Zn = Z + DZ;
        const int nx = fx_cell(Xn), ny = fx_cell(Yn), nz = fx_cell(Zn);
        const bool change = (nx != cx) | (ny != cy) | (nz != cz);
        const bool pf = change && k + 1 < k1;  // the next sample is interior and in a new cell
        float nxt[8], nxt2[8];
        if (pf) {
            s.template corners<false>(nx, ny, nz, nxt);
            if constexpr (TWO) s2.template corners<false>(nx, ny, nz, nxt2);
        }
        const float fx = fx_frac(X), fy = fx_frac(Y), fz = fx_frac(Z);
        float v = 0.0f;
        if constexpr (MODE == SHW_RATIO_MIP) {
            const float c1 = filter_value(trilerp(cur, fx, fy, fz), a), c2 = filter_value(trilerp(cur2, fx, fy, fz), a);
            st.update2(isnan(c1) ? a.lo : c1, isnan(c2) ? a.lo : c2);
        } else if constexpr (TWO) {
            // Algorithm 14: ratio where cube1 exceeds the floor, else DATAMIN
            const float c1 = filter_value(trilerp(cur, fx, fy, fz), a), c2 = filter_value(trilerp(cur2, fx, fy, fz), a);
            v = (c1 > a.ratio_floor) ? __fdiv_rn(c2, c1) : a.lo;
        } else {
            v = trilerp(cur, fx, fy, fz);
            v = filter_value(isnan(v) ? a.lo : v, a);
        }
        if constexpr (MODE != SHW_RATIO_MIP) {
            v = isnan(v) ? a.lo : v;  // a NaN sample counts as DATAMIN
            if (st.update(v, k)) {
                kdone = k + 1;
                return true;
            }
        }
        if (pf) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                cur[i] = nxt[i];
                if constexpr (TWO) cur2[i] = nxt2[i];
            }
            cx = nx;
            cy = ny;
            cz = nz;
        }
        X = Xn;
        Y = Yn;
        Z = Zn;
    }
    kdone = k1;
    return false;
}

// The interior loop for the sampler at hand.
template <int MODE, class S, class St>
__device__ __forceinline__ bool march_interior(const S &s, const S &s2, const RenderArgs &a, St &st, long long &X,
                                               long long &Y, long long &Z, long long DX, long long DY, long long DZ,
                                               int k0, int k1, int &kdone)
{
    if constexpr (S::kPair)
        return march_interior_pair<MODE>(s, a, st, X, Y, Z, DX, DY, DZ, k0, k1, kdone);
    else
        return march_interior_single<MODE>(s, s2, a, st, X, Y, Z, DX, DY, DZ, k0, k1, kdone);
}

// setFragment (Algorithm 1): the outputs of one ray from its final transfer-function
// state.  N: samples of the ray (0: it missed); P, D: its first sample and step (fixed
// point, x y z); done: samples processed.
template <int MODE, int INTERP, class St>
__device__ __forceinline__ void emit_ray(const RenderArgs &a, long long pix, int N, const long long P[3],
                                         const long long D[3], const St &st, int done)
{
    const long long PZ = P[2], DZ = D[2];
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    float scalar = 0.0f;
    int index = -1;
    if (N > 0) {
        if constexpr (MODE == SHW_MIP || MODE == kMipValue || MODE == SHW_SPECTRAL || MODE == SHW_RATIO) {
            const long long Zm = PZ + (long long)st.kmax * DZ;
            index = clampi(fx_round(Zm), 0, a.nz - 1);
            scalar = st.m;
            const float vh = normalise(st.m, a.lo, a.inv_range);
            if constexpr (MODE == SHW_SPECTRAL) {
                // Algorithm 4: colour from the spectral position, alpha from the value
                const float zmax =
                    (INTERP == SHW_NEAREST) ? (float)index : __ll2float_rn(Zm) * 2.3283064365386963e-10f;
                const float tz = __saturatef((zmax + 0.5f) / (float)a.nz);
                const float4 c = lut_eval(a.lut, tz);
                out = make_float4(c.x, c.y, c.z, colour_alpha(st.m, a));
            } else {
                out = lut_eval(a.lut, vh);
            }
        } else if constexpr (MODE == SHW_MIP_RGB) {
            // Algorithm 6: (r, g, b) = the maximum's (z, y, x) as texture coordinates
            const bool near = INTERP == SHW_NEAREST;
            const long long km = (long long)st.kmax;
            const float zm = colour_pos(PZ + km * DZ, a.nz, near);
            index = clampi(fx_round(PZ + km * DZ), 0, a.nz - 1);
            scalar = st.m;
            out = make_float4(tex_coord(zm, a.nz), tex_coord(colour_pos(P[1] + km * D[1], a.ny, near), a.ny),
                              tex_coord(colour_pos(P[0] + km * D[0], a.nx, near), a.nx), colour_alpha(st.m, a));
        } else if constexpr (MODE == SHW_RATIO_MIP) {
            // Algorithm 13: the colour of max2 / max1 where max1 passes the floor, else
            // transparent black
            scalar = a.lo;
            if (st.m1 > a.ratio_floor) {
                scalar = __fdiv_rn(st.m2, st.m1);
                out = lut_eval(a.lut, normalise(scalar, a.lo, a.inv_range));
            }
        } else if constexpr (MODE == SHW_AVG) {
            scalar = __fdiv_rn(st.sum, (float)N);
            out = lut_eval(a.lut, normalise(scalar, a.lo, a.inv_range));
        } else if constexpr (MODE == SHW_MOMENT1) {
            if (st.sw > 0.0f) {
                const float m1 = __fdiv_rn(st.szw, st.sw);
                scalar = m1;
                index = clampi(__float2int_rd(m1 + 0.5f), 0, a.nz - 1);
                const float tz = __saturatef((m1 + 0.5f) / (float)a.nz);
                const float4 c = lut_eval(a.lut, tz);
                out = make_float4(c.x, c.y, c.z, colour_alpha(__fdiv_rn(st.sv, (float)N), a));
            }
        } else {
            out = make_float4(st.cr, st.cg, st.cb, 1.0f - st.T);
            scalar = 1.0f - st.T;
        }
    } else {
        done = 0;
    }
    if constexpr (MODE == SHW_COMPOSITE)
        if (a.ckpt_K != nullptr) a.ckpt_K[pix] = done;
    a.rgba[pix] = out;
    if (a.scalar) a.scalar[pix] = scalar;
    if (a.index) a.index[pix] = index;
    if (a.nsamples) a.nsamples[pix] = done;
}

// The transfer-function state of one ray before its first sample (Algorithm 1's "init
// vars"): the colour map, opacity scale and checkpoint slots of compositing, the first
// sample's position for the position-coloured modes and the first moment.
template <int MODE, int INTERP, class St, class S>
__device__ __forceinline__ void init_ray_state(St &st, const S &s, const RenderArgs &a, const RayFx &r, long long pix,
                                               const float4 *lut_c)
{
    if constexpr (is_composite<MODE>) {
        st.lut = lut_c;
        st.lo = a.lo;
        st.inv_range = a.inv_range;
        st.s = a.opacity_scale;
        st.term = a.term_alpha;
        st.ckpt = a.ckpt_T != nullptr ? a.ckpt_T + pix : nullptr;
        st.ckpt_stride = (long long)a.width * a.height;
        st.I = a.ckpt_interval;
        st.nckpt = a.nckpt;
        if constexpr (MODE != SHW_COMPOSITE) {
            st.X = r.P[0];
            st.Y = r.P[1];
            st.Z = r.P[2];
            st.DX = r.D[0];
            st.DY = r.D[1];
            st.DZ = r.D[2];
            st.nx = s.nx;
            st.ny = s.ny;
            st.nz = s.nz;
            st.nearest = INTERP == SHW_NEAREST;
        }
    }
    if constexpr (MODE == SHW_MOMENT1) {
        st.Z = r.P[2];
        st.DZ = r.D[2];
        st.lo = a.lo;
        st.nz = a.nz;
        st.nearest = INTERP == SHW_NEAREST;
    }
}

// One ray of Algorithm 1 with the transfer function MODE.  lut_c: the colour map in
// shared memory (read per sample by COMPOSITE); a.lut: the same map in global memory.
// SMK: 0 no in-ray smoothing; 1 smoothing by direct fetches; 2 the box on the sample lattice
// (a step of 1/2 voxel, single-cube modes).
template <int MODE, int INTERP, class S, int SMK = 0>
__device__ __forceinline__ void render_pixel(const S &s, const S &s2, const shw_camera &cam, const RenderArgs &a,
                                             const float4 *lut_c, int px, int py)
{
    const long long pix = (long long)py * a.width + px;

    RayFx r;
    const bool hit = !quick_miss(cam, px, py, s.nx, s.ny, s.nz) && setup_ray(cam, px, py, s.nx, s.ny, s.nz, a.step, r);
    const int N = hit ? min(r.N, a.nmax) : 0;

    int done = 0;
    typename StateOf<MODE>::type st;
    if (N > 0) {
        int ka, kb;
        interior_range(r, s.nx, s.ny, s.nz, N, ka, kb);
        long long X = r.P[0], Y = r.P[1], Z = r.P[2];
        const long long DX = r.D[0], DY = r.D[1], DZ = r.D[2];
        init_ray_state<MODE, INTERP>(st, s, a, r, pix, lut_c);
        CacheOf<S> cc, cc2;
        if constexpr (SMK == 2) {
            march_box_lattice<2, MODE, INTERP>(s, a, st, r.P, r.D, N, done);
        } else if constexpr (SMK == 1) {
            // smoothing: taps reach past the interior, so every sample fetches with clamping
            march<true, MODE, INTERP, true>(s, s2, a, st, cc, cc2, X, Y, Z, DX, DY, DZ, 0, N, done, r.U);
        } else {
        bool stop = march<true, MODE, INTERP>(s, s2, a, st, cc, cc2, X, Y, Z, DX, DY, DZ, 0, ka, done);
        if (!stop) {
            // (16-bit bricks: only for the line ratio, whose two gathers per sample leave
            // the most latency to hide; otherwise the extra registers cost more)
            if constexpr (INTERP == SHW_TRILINEAR && SHW_PREFETCH && (S::kLinearF32 || two_cubes<MODE>)) {
                stop = march_interior<MODE>(s, s2, a, st, X, Y, Z, DX, DY, DZ, ka, kb, done);
                cc.ix = cc2.ix = -4;  // the tail starts with a fresh cell
            } else {
                stop = march<false, MODE, INTERP>(s, s2, a, st, cc, cc2, X, Y, Z, DX, DY, DZ, ka, kb, done);
            }
        }
        if (!stop) march<true, MODE, INTERP>(s, s2, a, st, cc, cc2, X, Y, Z, DX, DY, DZ, kb, N, done);
        }
    }
    if (N <= 0) r.P[0] = r.P[1] = r.P[2] = r.D[0] = r.D[1] = r.D[2] = 0;
    emit_ray<MODE, INTERP>(a, pix, N, r.P, r.D, st, done);
}

template <int MODE, int INTERP, class S>
__global__ void __launch_bounds__(kRenderThreads) render_kernel(S s, S s2, shw_camera cam, RenderArgs a)
{
    __shared__ float4 lut_s[kLut];
    const float4 *lut_c = a.lut;
    if constexpr (is_composite<MODE> && SHW_LUT_SMEM) {
        for (int i = threadIdx.x; i < kLut; i += blockDim.x) lut_s[i] = a.lut[i];
        __syncthreads();
        lut_c = lut_s;
    }
    int px, py;
    tile_pixel(px, py, a);
    if (px >= a.width || py >= a.height) return;
    render_pixel<MODE, INTERP, S>(s, s2, cam, a, lut_c, px, py);
}

#ifndef SHW_RENDER_PERSISTENT
#define SHW_RENDER_PERSISTENT 1  // 1: resident CTAs whose warps take warp tiles from a counter
#endif

// host: a zeroed work counter for one persistent launch on stream st (null on failure),
// and the device's SM count
unsigned *work_counter(cudaStream_t st);
int sm_count();

// Persistent form: every warp takes the next warp tile (centre-out order, as above)
// from a global counter until none is left, so no SM idles while rays of very
// different lengths finish and no CTA launch overhead is paid per tile.
#ifndef SHW_RENDER_MINB
#define SHW_RENDER_MINB 1  // minimum resident CTAs per SM the persistent kernel is compiled for
#endif
template <int MODE, int INTERP, class S, int SMK = 0>
__global__ void __launch_bounds__(kRenderThreads, SHW_RENDER_MINB)
    render_kernel_persistent(S s, S s2, shw_camera cam, RenderArgs a, unsigned *ctr, int nwarp_tiles)
{
    const int lane = threadIdx.x & 31;
    const int ws = a.warp_shift, wtx = 1 << ws, wty = 32 >> ws;
    int tw, th;
    cta_tile(ws, tw, th);
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(ctr, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned)nwarp_tiles) break;
        const int rank = (int)t / kCtaWarps, warp = (int)t - rank * kCtaWarps;
        const int rr = rank / a.tiles_x, cr = rank - rr * a.tiles_x;
        const int ty = centre_out(rr, a.cty, a.tiles_y), tx = centre_out(cr, a.ctx, a.tiles_x);
        const int px = tx * tw + (wtx >= wty ? 0 : warp * wtx) + (lane & (wtx - 1));
        const int py = ty * th + (wtx >= wty ? warp * wty : 0) + (lane >> ws);
        if (px < a.width && py < a.height) render_pixel<MODE, INTERP, S, SMK>(s, s2, cam, a, a.lut, px, py);
    }
}

// Resident CTAs per SM of one kernel, queried once per kernel (a static per instance).
template <auto KERN>
int resident_per_sm()
{
    static int per_sm = -1;
    if (per_sm < 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, KERN, kRenderThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        per_sm = n;
    }
    return per_sm;
}

// Pixel coordinates of the cube centre's projection (image centre if behind the eye).
inline void project_centre(const shw_camera &c, int nx, int ny, int nz, float &px, float &py)
{
    const float q[3] = {0.5f * (nx - 1) - c.eye[0], 0.5f * (ny - 1) - c.eye[1], 0.5f * (nz - 1) - c.eye[2]};
    const float r = q[0] * c.right[0] + q[1] * c.right[1] + q[2] * c.right[2];
    const float u = q[0] * c.up[0] + q[1] * c.up[1] + q[2] * c.up[2];
    const float f = q[0] * c.fwd[0] + q[1] * c.fwd[1] + q[2] * c.fwd[2];
    const float aspect = (float)c.width / (float)c.height;
    float xs = 0.0f, ys = 0.0f;
    if (c.ortho) {
        xs = r / (c.ortho_half_h * aspect);
        ys = u / c.ortho_half_h;
    } else if (f > 0.0f) {
        xs = r / (f * c.tan_half_fovy * aspect);
        ys = u / (f * c.tan_half_fovy);
    }
    px = 0.5f * (xs + 1.0f) * c.width;
    py = 0.5f * (1.0f - ys) * c.height;
}

// Host-side launch for one storage type (instantiated per storage in its own TU).
// SMK > 0: the in-ray smoothing instances (persistent form only; see render_pixel).
template <int SMK, class S>
shw_status launch_render_modes(int mode, int interp, const S &s, const S &s2, const shw_camera &cam,
                               const RenderArgs &a0, cudaStream_t st)
{
    RenderArgs a = a0;
    int tw, th;
    cta_tile(a.warp_shift, tw, th);
    a.tiles_x = ceil_div(cam.width, tw);
    a.tiles_y = ceil_div(cam.height, th);
    const long long tiles = (long long)a.tiles_x * a.tiles_y;
    float cpx, cpy;
    project_centre(cam, s.nx, s.ny, s.nz, cpx, cpy);
    a.ctx = (int)fminf(fmaxf(cpx / tw, 0.0f), (float)(a.tiles_x - 1));
    a.cty = (int)fminf(fmaxf(cpy / th, 0.0f), (float)(a.tiles_y - 1));
    const dim3 grid((unsigned)tiles);
    const dim3 block(kRenderThreads);
    unsigned *ctr = SHW_RENDER_PERSISTENT ? work_counter(st) : nullptr;
    const int nsm = sm_count();
    const int nwarp_tiles = (int)(tiles * kCtaWarps);
    // persistent grid: as many CTAs as fit on the device at once (at most one per tile)
    auto persistent = [&](auto kern, int per_sm) {
        const long long g = std::min<long long>((long long)per_sm * nsm, tiles);
        kern<<<(unsigned)std::max<long long>(g, 1), block, 0, st>>>(s, s2, cam, a, ctr, nwarp_tiles);
    };
    if (SMK > 0 && (ctr == nullptr || nsm <= 0)) return SHW_ECUDA;
#define SHW_LAUNCH(M, I)                                                       \
    do {                                                                       \
        if constexpr (SMK > 0)                                                 \
            persistent(render_kernel_persistent<M, I, S, SMK>,                 \
                       resident_per_sm<render_kernel_persistent<M, I, S, SMK>>()); \
        else if (ctr != nullptr && nsm > 0)                                    \
            persistent(render_kernel_persistent<M, I, S>,                      \
                       resident_per_sm<render_kernel_persistent<M, I, S>>());  \
        else                                                                   \
            render_kernel<M, I, S><<<grid, block, 0, st>>>(s, s2, cam, a);     \
    } while (0)
#define SHW_CASE(M)                                            \
    case M:                                                    \
        if (interp == SHW_NEAREST) SHW_LAUNCH(M, SHW_NEAREST); \
        else SHW_LAUNCH(M, SHW_TRILINEAR);                     \
        break;
    if constexpr (S::kPair) {
        // the interleaved pair storage serves the line ratios only
        switch (mode) {
            SHW_CASE(SHW_RATIO)
            SHW_CASE(SHW_RATIO_MIP)
        default:
            return SHW_EUNSUPPORTED;
        }
    } else if constexpr (SMK == 2) {
        // the lattice box: single-cube modes
        switch (mode) {
            SHW_CASE(SHW_MIP)
            SHW_CASE(SHW_AVG)
            SHW_CASE(SHW_COMPOSITE)
            SHW_CASE(SHW_SPECTRAL)
            SHW_CASE(SHW_MOMENT1)
            SHW_CASE(SHW_COMPOSITE_SPECTRAL)
            SHW_CASE(SHW_MIP_RGB)
            SHW_CASE(SHW_COMPOSITE_RGB)
        default:
            return SHW_EUNSUPPORTED;
        }
    } else {
    switch (mode) {
        SHW_CASE(SHW_MIP)
        SHW_CASE(SHW_AVG)
        SHW_CASE(SHW_COMPOSITE)
        SHW_CASE(SHW_SPECTRAL)
        SHW_CASE(SHW_RATIO)
        SHW_CASE(SHW_MOMENT1)
        SHW_CASE(SHW_COMPOSITE_SPECTRAL)
        SHW_CASE(SHW_MIP_RGB)
        SHW_CASE(SHW_COMPOSITE_RGB)
        SHW_CASE(SHW_RATIO_MIP)
    default:
        return SHW_EINVAL;
    }
    }
#undef SHW_CASE
#undef SHW_LAUNCH
    return after_launch();
}

// Warp tile orientation for a camera (see the layout note at the top).
inline int warp_shift_for(const shw_camera &c)
{
    if (SHW_WARP_SHIFT >= 0) return SHW_WARP_SHIFT;
    const float rx = c.right[0] < 0 ? -c.right[0] : c.right[0], ux = c.up[0] < 0 ? -c.up[0] : c.up[0];
    if (rx >= 0.5f && rx >= ux) return 4;
    if (ux >= 0.5f) return 1;
    return 3;
}

// Entry points of the per-storage translation units.
shw_status render_f32(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                      const RenderArgs &a, cudaStream_t st);
shw_status render_f32_big(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                          const RenderArgs &a, cudaStream_t st);
// the line ratios on the interleaved pair storages (any of SHW_F32_PAIR, SHW_*_PAIR_BRICK)
shw_status render_f32_pair(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                           cudaStream_t st);
shw_status render_pair(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                       cudaStream_t st);
// in-ray smoothing (a.smooth != SHW_SMOOTH_NONE), any storage; the _lat forms run the box on
// the sample lattice (a.box_lattice == 2)
shw_status render_smooth_f32(int mode, int interp, const shw_volume &v, const shw_volume *v2,
                             const shw_camera &cam, const RenderArgs &a, cudaStream_t st);
shw_status render_smooth_b16(int mode, int interp, const shw_volume &v, const shw_volume *v2,
                             const shw_camera &cam, const RenderArgs &a, cudaStream_t st);
shw_status render_smooth_lat_f32(int mode, int interp, const shw_volume &v, const shw_camera &cam,
                                 const RenderArgs &a, cudaStream_t st);
shw_status render_smooth_lat_b16(int mode, int interp, const shw_volume &v, const shw_camera &cam,
                                 const RenderArgs &a, cudaStream_t st);
shw_status render_bf16(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                       const RenderArgs &a, cudaStream_t st);
shw_status render_f16(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                      const RenderArgs &a, cudaStream_t st);
shw_status render_bf16_big(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                           const RenderArgs &a, cudaStream_t st);
shw_status render_f16_big(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                          const RenderArgs &a, cudaStream_t st);
// the staged marcher (render_slab.cu); SHW_EUNSUPPORTED if it does not apply
shw_status render_slab(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                       cudaStream_t st);
// the plane sweep for orthographic spectral-axis views (render_axis.cu); SHW_EUNSUPPORTED if it does not apply
shw_status render_axis(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                       cudaStream_t st);

}  // namespace shw
