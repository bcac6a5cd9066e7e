// render_impl.cuh -- the ray marcher: one thread per pixel (= one ray, the
// fragment of Section 2.3), Algorithm 1's loop with one transfer function.
//
// Thread layout: a CTA of 256 threads renders a 16 x 16 pixel tile; each warp
// owns an 8 x 4 sub-tile so that its 32 rays stay close in 3-D and their loads
// share cache lines.
#pragma once

#include <cuda_runtime.h>

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
    int nmax;  // upper bound of N over all rays (box diagonal / step + 1)
    int warp_shift;
    float step, lo, inv_range, opacity_scale, term_alpha, ratio_floor;
    int nz;
};

constexpr int kTileX = 16, kTileY = 16, kRenderThreads = 256;
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
    return make_float4(lerp(a.x, b.x, f), lerp(a.y, b.y, f), lerp(a.z, b.z, f), lerp(a.w, b.w, f));
}

__device__ __forceinline__ float normalise(float v, float lo, float inv_range)
{
    // fmaxf first: a NaN argument yields 0 (never reached: NaN samples become lo)
    return fminf(fmaxf((v - lo) * inv_range, 0.0f), 1.0f);
}

// Pixel of this thread.  A warp covers a (2^ws) x (32 / 2^ws) pixel tile: ws = 4 (16 x 2)
// or 1 (2 x 16) when rows or columns of the image run close to the cube's x axis
// (the contiguous one, so a warp's loads share cache lines), ws = 3 (8 x 4) otherwise.
__device__ __forceinline__ void tile_pixel(int &px, int &py, int ws)
{
    const int wtx = 1 << ws, wty = 32 >> ws, wpr = kTileX >> ws;  // warps per tile row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    px = blockIdx.x * kTileX + (warp % wpr) * wtx + (lane & (wtx - 1));
    py = blockIdx.y * kTileY + (warp / wpr) * wty + (lane >> ws);
}

template <int INTERP, class S>
__device__ __forceinline__ float fetch(const S &s, long long X, long long Y, long long Z)
{
    if constexpr (INTERP == SHW_NEAREST)
        return s.nearest(X, Y, Z);
    else
        return s.trilinear(X, Y, Z);
}

// the marcher's fetch: with SHW_CELL_CACHE, trilinear samples reuse the previous cell's corners
template <int INTERP, class S>
__device__ __forceinline__ float fetch_c(const S &s, long long X, long long Y, long long Z, CellCache &cc)
{
    if constexpr (INTERP == SHW_TRILINEAR && SHW_CELL_CACHE)
        return trilinear_cached(s, X, Y, Z, cc);
    else
        return fetch<INTERP>(s, X, Y, Z);
}

// One ray of Algorithm 1 with the transfer function MODE.  lut_c: the colour map in
// shared memory (read per sample by COMPOSITE); a.lut: the same map in global memory.
template <int MODE, int INTERP, class S>
__device__ __forceinline__ void render_pixel(const S &s, const S &s2, const shw_camera &cam, const RenderArgs &a,
                                             const float4 *lut_c, int px, int py)
{
    const long long pix = (long long)py * a.width + px;
    const long long npix = (long long)a.width * a.height;

    RayFx r;
    const bool hit = setup_ray(cam, px, py, s.nx, s.ny, s.nz, a.step, r);
    const int N = hit ? min(r.N, a.nmax) : 0;

    long long X = r.P[0], Y = r.P[1], Z = r.P[2];
    const long long DX = r.D[0], DY = r.D[1], DZ = r.D[2];

    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    float scalar = 0.0f;
    int index = -1;
    int done = 0;

    if constexpr (MODE == SHW_MIP || MODE == SHW_SPECTRAL || MODE == SHW_RATIO) {
        float m = -INFINITY;
        int kmax = 0;
        CellCache cc, cc2;
        for (int k = 0; k < N; ++k) {
            float v;
            if constexpr (MODE == SHW_RATIO) {
                // Algorithm 14: ratio where cube1 exceeds the floor, else DATAMIN
                const float c1 = fetch_c<INTERP>(s, X, Y, Z, cc), c2 = fetch_c<INTERP>(s2, X, Y, Z, cc2);
                v = (c1 > a.ratio_floor) ? __fdiv_rn(c2, c1) : a.lo;
            } else {
                v = fetch_c<INTERP>(s, X, Y, Z, cc);
            }
            v = isnan(v) ? a.lo : v;
            if (v >= m) {  // Eq. 1: ">=", the last maximum along the ray wins
                m = v;
                kmax = k;
            }
            X += DX;
            Y += DY;
            Z += DZ;
        }
        done = N;
        if (N > 0) {
            const long long Zm = r.P[2] + (long long)kmax * DZ;
            index = clampi(fx_round(Zm), 0, a.nz - 1);
            scalar = m;
            const float vh = normalise(m, a.lo, a.inv_range);
            if constexpr (MODE == SHW_SPECTRAL) {
                // Algorithm 4: colour from the spectral position, alpha from the value
                const float zmax = (INTERP == SHW_NEAREST) ? (float)index : __ll2float_rn(Zm) * 2.3283064365386963e-10f;
                const float tz = fminf(fmaxf((zmax + 0.5f) / (float)a.nz, 0.0f), 1.0f);
                const float4 c = lut_eval(a.lut, tz);
                out = make_float4(c.x, c.y, c.z, vh);
            } else {
                out = lut_eval(a.lut, vh);
            }
        }
    } else if constexpr (MODE == SHW_AVG) {
        // Eq. 3 divided by N; compensated (Kahan) summation keeps FP32 exact enough
        float sum = 0.0f, comp = 0.0f;
        CellCache cc;
        for (int k = 0; k < N; ++k) {
            float v = fetch_c<INTERP>(s, X, Y, Z, cc);
            v = isnan(v) ? a.lo : v;
            const float y = __fsub_rn(v, comp);
            const float t = __fadd_rn(sum, y);
            comp = __fsub_rn(__fsub_rn(t, sum), y);
            sum = t;
            X += DX;
            Y += DY;
            Z += DZ;
        }
        done = N;
        if (N > 0) {
            scalar = __fdiv_rn(sum, (float)N);
            out = lut_eval(a.lut, normalise(scalar, a.lo, a.inv_range));
        }
    } else {  // SHW_COMPOSITE: Algorithm 3 in premultiplied form
        float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        const int I = a.ckpt_interval;
        int k = 0;
        CellCache cc;
        for (; k < N;) {
            if (a.ckpt_T != nullptr && (k % I) == 0 && k / I < a.nckpt) a.ckpt_T[(long long)(k / I) * npix + pix] = T;
            float v = fetch_c<INTERP>(s, X, Y, Z, cc);
            v = isnan(v) ? a.lo : v;
            const float4 c = lut_eval(lut_c, normalise(v, a.lo, a.inv_range));
            const float al = fminf(fmaxf(a.opacity_scale * c.w, 0.0f), 1.0f);
            const float w = T * al;
            cr = __fmaf_rn(w, c.x, cr);
            cg = __fmaf_rn(w, c.y, cg);
            cb = __fmaf_rn(w, c.z, cb);
            T = T * (1.0f - al);
            ++k;
            if (1.0f - T > a.term_alpha) break;  // early ray termination
            X += DX;
            Y += DY;
            Z += DZ;
        }
        done = k;
        out = make_float4(cr, cg, cb, 1.0f - T);
        scalar = 1.0f - T;
        if (a.ckpt_K != nullptr) a.ckpt_K[pix] = k;
    }

    a.rgba[pix] = out;
    if (a.scalar) a.scalar[pix] = scalar;
    if (a.index) a.index[pix] = index;
    if (a.nsamples) a.nsamples[pix] = done;
}

template <int MODE, int INTERP, class S>
__global__ void __launch_bounds__(kRenderThreads) render_kernel(S s, S s2, shw_camera cam, RenderArgs a)
{
    __shared__ float4 lut_s[kLut];
    if constexpr (MODE == SHW_COMPOSITE) {
        for (int i = threadIdx.x; i < kLut; i += blockDim.x) lut_s[i] = a.lut[i];
        __syncthreads();
    }
    int px, py;
    tile_pixel(px, py, a.warp_shift);
    if (px >= a.width || py >= a.height) return;
    render_pixel<MODE, INTERP, S>(s, s2, cam, a, lut_s, px, py);
}

// Host-side launch for one storage type (instantiated per storage in its own TU).
template <class S>
shw_status launch_render_modes(int mode, int interp, const S &s, const S &s2, const shw_camera &cam,
                               const RenderArgs &a, cudaStream_t st)
{
    const dim3 grid((unsigned)ceil_div(cam.width, kTileX), (unsigned)ceil_div(cam.height, kTileY));  // height <= 2^19
    const dim3 block(kRenderThreads);
#define SHW_LAUNCH(M, I) render_kernel<M, I, S><<<grid, block, 0, st>>>(s, s2, cam, a)
#define SHW_CASE(M)                                          \
    case M:                                                  \
        if (interp == SHW_NEAREST) SHW_LAUNCH(M, SHW_NEAREST); \
        else SHW_LAUNCH(M, SHW_TRILINEAR);                   \
        break;
    switch (mode) {
        SHW_CASE(SHW_MIP)
        SHW_CASE(SHW_AVG)
        SHW_CASE(SHW_COMPOSITE)
        SHW_CASE(SHW_SPECTRAL)
        SHW_CASE(SHW_RATIO)
    default:
        return SHW_EINVAL;
    }
#undef SHW_CASE
#undef SHW_LAUNCH
    return after_launch();
}

// Warp tile orientation for a camera (see tile_pixel).
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
shw_status render_bf16(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                       const RenderArgs &a, cudaStream_t st);
shw_status render_f16(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                      const RenderArgs &a, cudaStream_t st);

}  // namespace shw
